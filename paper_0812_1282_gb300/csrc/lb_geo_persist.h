// Host entry points of the multi-step obstacle steps (lb_geo.cu).
#pragma once

#include "lb_internal.h"

namespace lbfe {

// Persistent multi-step obstacle step (a cooperative launch of one CTA per
// tile for n_steps steps, step s reading buffer parity0 ^ (s & flip));
// flags: geo_tiles(nx, ny) ints, done: one int, all zero between launches.
// geo_persist_occupancy: resident CTAs per SM (0 on error).
int geo_tiles(int nx, int ny);
int geo_persist_occupancy(int precision, int coll);
int launch_geo_persist(int precision, int coll, const DomDesc& d, int parity0, int flip,
                       int n_steps, int* flags, int* done, void* stream);
// Two steps of an obstacle domain in one launch (temporal blocking): reads
// buffer `parity`, writes the other (which then holds the state two steps
// on).  prepare_geo_step2 opts the kernel in to its shared memory (once per
// device, outside any stream capture).
int launch_geo_step2(int precision, int coll, const DomDesc& d, int parity, void* stream);
int prepare_geo_step2();

}  // namespace lbfe
