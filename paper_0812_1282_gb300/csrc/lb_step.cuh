// Fused stream + collide time step (Steps 1-4 of Sec. V, pull form),
// staged through shared memory by asynchronous bulk copies (TMA) in a
// warp-specialised producer / consumer pipeline.
//
// A CTA owns a strip of W = 32 * NW columns and marches up through `rows`
// lattice rows.  Warp 0 is the producer: for every lattice row r the strip
// touches it issues, from 18 lanes at once, the 18 bulk copies
// (cp.async.bulk) of the plane-row segments that the pull of row r reads:
// for direction i the segment of plane i at row r - e_iy (or plane opp(i)
// at row r for a bounce-back link), columns x0-4 .. x0+W+4.  A stage thus
// holds exactly the 9 f and 9 g values every node of row r pulls, at column
// offsets -1/0/+1 (the two rows just outside the tile are only read for
// their phi, so only their 9 g segments are copied).  Stages live in an
// S-slot ring; slot k has a "full"
// mbarrier (completed by the copies' transaction bytes) and an "empty"
// mbarrier (one arrival per compute warp that is done with it).
//
// Warps 1..NW compute; warp w owns 32 columns, one node per lane per row,
// and runs independently of the other compute warps:
//   1. wait until the stage of row y+1 is full, compute phi there for its 32
//      columns and (lanes 0 / 31) the two halo columns, into a warp-private
//      4-row ring of phi values (wetting ghost rows outside the walls);
//   2. read f and g of row y from its stage, take the 3x3 phi stencil from
//      the ring, collide, store 18 values, and release the stage.
// Nothing but the stage ring couples the warps, so no CTA-wide barrier sits
// in the row loop.
//
// Storage layout (see lb_internal.h): logical column x lives at physical
// column x + kXOff of each row; physical columns kXOff-2, kXOff-1 hold copies
// of logical nx-2, nx-1 and physical nx+kXOff, nx+kXOff+1 hold copies of
// logical 0, 1 (periodic ghosts, written by the step itself), so every
// segment is one contiguous, 16-byte aligned copy for any nx.
//
// Pull rule (Eqs. stream1-2 and mid-link bounce-back): f_i(r) =
// f'_i(r - e_i), or f'_opp(i)(r) when r - e_i is inside a wall.
#pragma once

#include "lb_async.cuh"
#include "lb_internal.h"
#include "lb_node.cuh"

namespace lbfe {

template <typename Real>
__device__ __forceinline__ NodeParams<Real> node_params(const DomDesc& D);
template <>
__device__ __forceinline__ NodeParams<float> node_params<float>(const DomDesc& D)
{
    return NodeParams<float>{D.fa,      D.fkappa,  D.fgamma,   D.fomega_phi,
                             D.ftau_c0, D.ftau_c1, D.fh_bot,   D.fh_top,
                             D.flut_lo, D.flut_step, D.flut_inv, D.flut_kmax};
}
template <>
__device__ __forceinline__ NodeParams<double> node_params<double>(const DomDesc& D)
{
    return NodeParams<double>{D.a,      D.kappa,  D.gamma,   D.omega_phi,
                              D.tau_c0, D.tau_c1, D.h_bot,   D.h_top,
                              D.lut_lo, D.lut_step, D.lut_inv, D.lut_kmax};
}

// velocity y-components in the paper's order, and the opposite direction
__device__ __forceinline__ int ey_of(int i)
{
    return (i == 3 || i == 5 || i == 7) ? 1 : ((i == 4 || i == 6 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Read the nine pulled values of the node at segment index c from a stage
// part (9 segments of width segw).  blo / bhi: the row sits on the bottom /
// top wall, so the links from below / above bounce back (their segments hold
// the opposite plane of the same row, read at the node's own column).
template <typename Real>
__device__ __forceinline__ void read9(const Real* __restrict__ s, int segw, int c, bool blo,
                                      bool bhi, Real (&v)[9])
{
    v[0] = s[0 * segw + c];
    v[1] = s[1 * segw + c - 1];
    v[2] = s[2 * segw + c + 1];
    v[3] = s[3 * segw + c];
    v[4] = s[4 * segw + c];
    v[5] = s[5 * segw + (blo ? c : c - 1)];
    v[6] = s[6 * segw + (bhi ? c : c + 1)];
    v[7] = s[7 * segw + (blo ? c : c + 1)];
    v[8] = s[8 * segw + (bhi ? c : c - 1)];
}

// Shared-memory carve-up for one CTA of NW compute warps (byte offsets):
// S full + S empty mbarriers, S stages of 18 segments of W + 8 elements,
// and one 4-row ring of 34 phi values per compute warp.
template <typename Real>
struct StageLayout {
    int NW, S, W, segw;
    __host__ __device__ StageLayout(int nw, int s) : NW(nw), S(s), W(32 * nw), segw(32 * nw + 8) {}
    __host__ __device__ size_t full() const { return 0; }
    __host__ __device__ size_t empty() const { return 64; }
    __host__ __device__ size_t stages() const { return 128; }
    __host__ __device__ size_t stage_elems() const { return size_t(18) * segw; }
    __host__ __device__ size_t rings() const
    {
        return stages() + size_t(S) * stage_elems() * sizeof(Real);
    }
    __host__ __device__ size_t total() const
    {
        return rings() + size_t(NW) * 4 * 34 * sizeof(Real);
    }
};

// Rows a tile stages: first .. last (wrapped when y is periodic).
struct TileRows {
    int first, last, y1;
    __device__ __forceinline__ TileRows(int y0, int rows, int ny, bool walls)
    {
        y1 = min(y0 + rows, ny);
        first = (walls && y0 == 0) ? 0 : y0 - 1;
        last = (walls && y1 == ny) ? ny - 1 : y1;
    }
    __device__ __forceinline__ int count() const { return last - first + 1; }
};

// ----------------------------------------------------------- producer
// Warp 0: issue the stages of one tile.  q counts the stages this CTA has
// issued so far (it continues across tiles of a persistent CTA).
template <typename Real, int S, int NWC = 0>
__device__ __forceinline__ void produce_tile(const DomDesc& D, int parity, int x0, int y0, int rows,
                                             unsigned char* __restrict__ smem, int nw, unsigned& q,
                                             int* tags = nullptr, int tag = 0)
{
    const int NW = NWC > 0 ? NWC : nw;  // compile-time strip width when specialised
    const Real* __restrict__ fs = static_cast<const Real*>(parity ? D.f[1] : D.f[0]);
    const Real* __restrict__ gs = static_cast<const Real*>(parity ? D.g[1] : D.g[0]);
    const int ny = D.ny, pitch = D.pitch;
    const size_t P = size_t(D.plane);
    const bool walls = D.walls != 0;
    const StageLayout<Real> L(NW, S);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    Real* stage = reinterpret_cast<Real*>(smem + L.stages());
    const int lane = threadIdx.x & 31;
    const TileRows T(y0, rows, ny, walls);
    const int segw = L.segw;
    const int seglen = min(segw, pitch - x0);
    const uint32_t segbytes = uint32_t(seglen) * uint32_t(sizeof(Real));
    // lane l < 18 copies part l: f (l < 9) or g (l >= 9) of direction l % 9
    const int i = lane % 9;
    const int ey = ey_of(i);
    const Real* src_base = lane < 9 ? fs : gs;
    for (int p = 0; p < T.count(); ++p, ++q) {
        const unsigned slot = q % unsigned(S);
        const unsigned use = q / unsigned(S);
        // the slot's previous use must be released by every compute warp
        if (use > 0) mbar_wait_idle(empty + slot, (use - 1) & 1u, D.err);
        int r = T.first + p;
        r = r < 0 ? r + ny : (r >= ny ? r - ny : r);
        // rows y0-1 and y1 serve only the phi look-ahead: g segments only
        const bool g_only = (p == 0 && T.first < y0) || (p == T.count() - 1 && T.last >= T.y1);
        if (lane == 0) {
            // a persistent CTA names the tile in the slot of its first stage;
            // the arrive below (release) publishes it to the compute warps
            if (tags && p == 0) tags[slot] = tag;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(full + slot, (g_only ? 9u : 18u) * segbytes);
        }
        __syncwarp();
        if (lane < 18 && !(g_only && lane < 9)) {
            const bool blo = walls && r == 0, bhi = walls && r == ny - 1;
            int pl = i, rr;
            if ((ey > 0 && blo) || (ey < 0 && bhi)) {
                pl = opp_of(i);
                rr = r;
            } else {
                rr = r - ey;
                rr = rr < 0 ? rr + ny : (rr >= ny ? rr - ny : rr);
            }
            const Real* src = src_base + size_t(pl) * P + size_t(rr) * pitch + x0;
            Real* dst = stage + size_t(slot) * L.stage_elems() + size_t(lane) * segw;
            bulk_g2s(dst, src, segbytes, full + slot);
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------- consumer
// Compute warp cw (0-based among compute warps) processes its 32 columns of
// one tile.  q: stage sequence number of the tile's first stage.
// prm_shared, when set, holds the node parameters in shared memory; the
// collision then reads them at each use instead of keeping them in
// registers for the whole tile.
template <typename Real, bool MRT, int S, int NWC = 0>
__device__ __forceinline__ void consume_tile(const DomDesc& D, int parity, int x0, int y0, int rows,
                                             unsigned char* __restrict__ smem, int nw, int cw,
                                             unsigned& q,
                                             const NodeParams<Real>* prm_shared = nullptr)
{
    const int NW = NWC > 0 ? NWC : nw;  // compile-time strip width when specialised
    Real* __restrict__ fd = static_cast<Real*>(parity ? D.f[0] : D.f[1]);
    Real* __restrict__ gd = static_cast<Real*>(parity ? D.g[0] : D.g[1]);
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const int P = static_cast<int>(D.plane);
    const bool walls = D.walls != 0;
    const NodeParams<Real> prm = node_params<Real>(D);
    const StageLayout<Real> L(NW, S);
    const int segw = L.segw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    const Real* stage = reinterpret_cast<const Real*>(smem + L.stages());
    Real* ring = reinterpret_cast<Real*>(smem + L.rings()) + cw * 4 * 34;

    const int lane = threadIdx.x & 31;
    const TileRows T(y0, rows, ny, walls);
    const unsigned qb = q;
    q += unsigned(T.count());

    const int wx0 = x0 + 32 * cw;          // first column of this warp
    const int wcols = min(32, nx - wx0);   // may be <= 0 for a ragged tile
    const bool active = lane < wcols;
    const int x = wx0 + lane;
    const int ci = 32 * cw + lane + 4;     // segment index of the lane's column
    const bool left = lane == 0;
    const bool right = lane == wcols - 1;
    const int cl = 32 * cw + 3, cr = 32 * cw + wcols + 4;  // halo columns
    const int own = lane + 1, hr = wcols + 1;

    auto slot_of = [&](int p) { return (qb + unsigned(p)) % unsigned(S); };
    auto stage_ptr = [&](int p) { return stage + size_t(slot_of(p)) * L.stage_elems(); };
    auto wait_full = [&](int p) {
        const unsigned qq = qb + unsigned(p);
        mbar_wait(full + (qq % unsigned(S)), (qq / unsigned(S)) & 1u, D.err);
    };
    auto release = [&](int p) {
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + slot_of(p));
    };
    auto rslot = [&](int y) -> Real* { return ring + ((y - y0 + 1) & 3) * 34; };
    auto wrap_row = [&](int r) { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };
    // phi of lattice row r (staged at position p) into the ring slot of row ys
    auto publish = [&](int p, int r, int ys) {
        const Real* sg = stage_ptr(p) + 9 * segw;
        const bool blo = walls && r == 0, bhi = walls && r == ny - 1;
        Real* s = rslot(ys);
        Real v[9];
        read9<Real>(sg, segw, ci, blo, bhi, v);
        s[own] = phi_sum<Real>(v);
        if (left) {
            read9<Real>(sg, segw, cl, blo, bhi, v);
            s[0] = phi_sum<Real>(v);
        }
        if (right) {
            read9<Real>(sg, segw, cr, blo, bhi, v);
            s[hr] = phi_sum<Real>(v);
        }
    };
    auto ghost_row = [&](int yg, int ys, Real h2) {
        Real* sg = rslot(yg);
        const Real* ss = rslot(ys);
        sg[own] = ss[own] - h2;
        if (left) sg[0] = ss[0] - h2;
        if (right) sg[hr] = ss[hr] - h2;
    };

    const int first = T.first, y1 = T.y1;
    const bool bottom_ghost = walls && y0 == 0;
    // prologue: phi of rows y0-1 (or its ghost) and y0; a stage with no node
    // row of this tile (row y0-1) is released as soon as phi is read from it
    if (!bottom_ghost) {
        wait_full(0);
        if (active) publish(0, wrap_row(y0 - 1), y0 - 1);
        release(0);
    }
    wait_full(y0 - first);
    if (active) publish(y0 - first, y0, y0);
    if (bottom_ghost) {
        wait_full(1);
        if (active) {
            publish(1, 1, 1);
            // each lane forms its own entries: row k - 1 less k h (k = 2:
            // mirror about row 0; k = 1: one-sided across the wall plane)
            ghost_row(-1, D.wet_k - 1, Real(D.wet_k) * prm.h_bot);
        }
    }
    bool have_next = bottom_ghost;
    for (int y = y0; y < y1; ++y) {
        const int yn = y + 1;
        if (!have_next) {
            if (yn < ny || !walls) {
                wait_full(yn - first);
                if (active) publish(yn - first, wrap_row(yn), yn);
            } else if (active) {
                ghost_row(yn, ny - D.wet_k, Real(D.wet_k) * prm.h_top);
            }
        }
        have_next = false;
        __syncwarp();
        const int py = y - first;
        if (active) {
            const bool blo = walls && y == 0, bhi = walls && y == ny - 1;
            const Real* sb = stage_ptr(py);
            Real f[9], g[9];
            read9<Real>(sb, segw, ci, blo, bhi, f);
            read9<Real>(sb + 9 * segw, segw, ci, blo, bhi, g);
            const Real* sm = rslot(y - 1);
            const Real* sc = rslot(y);
            const Real* sp = rslot(y + 1);
            const Real c = sc[own];
            Real dx, dy, lap;
            stencils<Real>(c, sc[own + 1], sc[own - 1], sp[own], sm[own], sp[own + 1],
                           sp[own - 1], sm[own + 1], sm[own - 1], dx, dy, lap);
            const bool s2 = D.step2 && (blo || bhi);
            Real fo[9], go[9];
            if (prm_shared) {
                const volatile NodeParams<Real>& PV = *prm_shared;
                collide<Real, MRT>(PV, f, g, c, dx, dy, lap, s2, D.step2_relax_j != 0, fo, go);
            } else {
                collide<Real, MRT>(prm, f, g, c, dx, dy, lap, s2, D.step2_relax_j != 0, fo, go);
            }
            const int o = y * pitch + x + kXOff;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                fd[i * P + o] = fo[i];
                gd[i * P + o] = go[i];
            }
            // periodic ghost copies: logical 0, 1 also at nx, nx+1 and
            // logical nx-2, nx-1 also at -2, -1
            if (x < 2) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    fd[i * P + o + nx] = fo[i];
                    gd[i * P + o + nx] = go[i];
                }
            }
            if (x >= nx - 2) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    fd[i * P + o - nx] = fo[i];
                    gd[i * P + o - nx] = go[i];
                }
            }
        }
        release(py);
    }
    // the last staged row (look-ahead only) is released here
    if (T.last >= y1 && !(walls && y1 == ny)) release(T.count() - 1);
}

// Producer: the work list is exhausted; complete the next stage slot with
// no bytes and the tag -1, which tells the compute warps to stop.
template <typename Real, int S, int NWC = 0>
__device__ __forceinline__ void produce_end(unsigned char* smem, int nw, unsigned& q, int* tags,
                                            unsigned* err)
{
    const int NW = NWC > 0 ? NWC : nw;
    const StageLayout<Real> L(NW, S);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    const unsigned slot = q % unsigned(S), use = q / unsigned(S);
    if (use > 0) mbar_wait_idle(empty + slot, (use - 1) & 1u, err);
    if ((threadIdx.x & 31) == 0) {
        tags[slot] = -1;
        mbar_arrive(full + slot);
    }
    __syncwarp();
    ++q;
}

// Compute warps: wait for the first stage of the next tile and read its tag.
template <typename Real, int S, int NWC = 0>
__device__ __forceinline__ int next_tag(unsigned char* smem, int nw, unsigned q, const int* tags,
                                        unsigned* err)
{
    const int NW = NWC > 0 ? NWC : nw;
    const StageLayout<Real> L(NW, S);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    if (!mbar_wait(full + (q % unsigned(S)), (q / unsigned(S)) & 1u, err)) return -1;
    return *reinterpret_cast<const volatile int*>(tags + (q % unsigned(S)));
}

template <typename Real, int S, int NWC = 0>
__device__ __forceinline__ void init_stages(unsigned char* smem, int nw)
{
    const int NW = NWC > 0 ? NWC : nw;
    const StageLayout<Real> L(NW, S);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(full + k, 1);
            mbar_init(empty + k, NW);
        }
        fence_mbar_init();
    }
    __syncthreads();
}

// Before the producer warp exits, every bulk copy it issued must have
// landed (they all have unless a wait timed out; this bounded wait covers
// that case).
template <typename Real, int S, int NWC = 0>
__device__ __forceinline__ void drain_stages(unsigned char* smem, int nw, unsigned q,
                                             unsigned* err)
{
    const int NW = NWC > 0 ? NWC : nw;
    if (threadIdx.x != 0 || q == 0) return;
    const StageLayout<Real> L(NW, S);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    const unsigned n = q < unsigned(S) ? q : unsigned(S);
    for (unsigned k = 0; k < n; ++k) {
        const unsigned qq = q - 1 - k;  // last use of slot qq % S
        mbar_wait_idle(full + (qq % unsigned(S)), (qq / unsigned(S)) & 1u, err);
    }
}

}  // namespace lbfe
