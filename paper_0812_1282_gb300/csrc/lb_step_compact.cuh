// Fused step with compact g storage (FP32, tau_phi = 1).
//
// With tau_phi = 1 the post-collision g of a node is its equilibrium
// (Eq. gevo), so g'_1..g'_8 follow from four numbers of that node: phi, the
// mobility-weighted chemical potential G = Gamma mu and the equilibrium
// velocity u_eq (Appendix A).  The compact state keeps exactly those:
//   c0  phi as a 32-bit fixed-point word (2^-29, as the full form's g_0),
//   c1  G,  c2 u_eq,x,  c3 u_eq,y,
// and g'_0 = phi - sum_{i>0} g'_i implicitly.  A step then reads and writes
// 9 f + 4 values per node (104 bytes) instead of 9 f + 9 g (144).
//
// The order parameter of the next step follows from the pull rule
// (Eqs. stream1-2, mid-link bounce-back):
//   phi(r, t+1) = g'_0(r) + sum_{i>0} g'_i(r - e_i)
//               = phi(r, t) + [sum_{i>0} g'_i(r - e_i) - sum_{i>0} g'_i(r)],
// advanced as an exact integer add of the quantised bracket on the word.
//
// Pipeline (as the full-storage step, lb_step.cuh): warp 0 copies, for
// stage p of a tile, the 9 pulled f segments of row y and the 4 compact
// segments of row y + 2 (rows above and below the tile get compact-only
// stages).  Each compute warp
//   1. expands the compact row it receives into the 8 outgoing g'_i, their
//      sum and the phi word, for its 32 columns and two halo columns on each
//      side, into a warp-private 3-row ring;
//   2. forms phi(t+1) of row y + 1 from that ring (its 32 columns and one
//      halo column each side, all alike) into its 4-row phi ring;
//   3. collides row y (f from the stage, the phi stencil from the ring) and
//      stores 9 f and the node's new compact values.
// Each stage is consumed within one iteration, so a 3-slot stage ring keeps
// two rows of copies in flight.
#pragma once

#include "lb_async.cuh"
#include "lb_internal.h"
#include "lb_node.cuh"
#include "lb_step.cuh"

namespace lbfe {

constexpr int kStagesC = 3;    // stage-ring depth of the compact step
constexpr int kECols = 36;     // expanded columns per warp: 32 + 2 halo each side
constexpr int kEArrays = 10;   // phi word, g'_1..g'_8, sum of g'_1..g'_8
constexpr int kESlots = 3;     // expanded rows kept per warp

// Shared memory of one CTA (byte offsets): barriers, S stages of 13
// segments, then per compute warp the expanded-row ring and the phi ring.
struct StageLayoutC {
    int NW, S, W, segw;
    __host__ __device__ StageLayoutC(int nw, int s) : NW(nw), S(s), W(32 * nw), segw(32 * nw + 8)
    {
    }
    __host__ __device__ size_t full() const { return 0; }
    __host__ __device__ size_t empty() const { return 64; }
    __host__ __device__ size_t stages() const { return 128; }
    __host__ __device__ size_t stage_elems() const { return size_t(13) * segw; }
    __host__ __device__ size_t erings() const { return stages() + size_t(S) * stage_elems() * 4; }
    __host__ __device__ size_t ering_elems() const { return size_t(kESlots) * kEArrays * kECols; }
    __host__ __device__ size_t prings() const { return erings() + size_t(NW) * ering_elems() * 4; }
    __host__ __device__ size_t wrings() const { return prings() + size_t(NW) * 4 * 34 * 4; }
    __host__ __device__ size_t total() const { return wrings() + size_t(NW) * 34 * 4; }
};

// Stages of one tile: npro compact-only stages for the compact rows
// clo .. min(y0 + 1, chi), then one stage per tile row y with the f of row
// y and the compact row y + 2 when y + 2 <= chi.  Rows are logical (not
// wrapped); with walls they are clipped to the lattice.
struct TilePlanC {
    int y0, y1, clo, chi, npro;
    __device__ __forceinline__ TilePlanC(int y0_, int rows, int ny, bool walls)
    {
        y0 = y0_;
        y1 = min(y0 + rows, ny);
        clo = y0 - 2;
        chi = y1 + 1;
        if (walls) {
            clo = max(clo, 0);
            chi = min(chi, ny - 1);
        }
        npro = min(y0 + 1, chi) - clo + 1;
    }
    __device__ __forceinline__ int count() const { return npro + (y1 - y0); }
};

// ----------------------------------------------------------- producer
template <int S, int NWC = 0>
__device__ __forceinline__ void produce_tile_c(const DomDesc& D, int parity, int x0, int y0,
                                               int rows, unsigned char* __restrict__ smem, int nw,
                                               unsigned& q, int* tags = nullptr, int tag = 0)
{
    const int NW = NWC > 0 ? NWC : nw;
    const float* __restrict__ fs = static_cast<const float*>(parity ? D.f[1] : D.f[0]);
    const float* __restrict__ cs = static_cast<const float*>(parity ? D.g[1] : D.g[0]);
    const int ny = D.ny, pitch = D.pitch;
    const size_t P = size_t(D.plane);
    const bool walls = D.walls != 0;
    const StageLayoutC L(NW, S);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    float* stage = reinterpret_cast<float*>(smem + L.stages());
    const int lane = threadIdx.x & 31;
    const TilePlanC T(y0, rows, ny, walls);
    const int segw = L.segw;
    const int seglen = min(segw, pitch - x0);
    const uint32_t segbytes = uint32_t(seglen) * 4u;
    const int i = lane % 9;
    const int ey = ey_of(i);
    auto wrap_row = [&](int r) { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };
    for (int p = 0; p < T.count(); ++p, ++q) {
        const unsigned slot = q % unsigned(S);
        const unsigned use = q / unsigned(S);
        if (use > 0) mbar_wait(empty + slot, (use - 1) & 1u, D.err);
        const int yf = p < T.npro ? -1 : y0 + (p - T.npro);          // f row (or none)
        const int ycl = p < T.npro ? T.clo + p : yf + 2;             // compact row (logical)
        const bool has_f = yf >= 0, has_c = ycl <= T.chi;
        if (lane == 0) {
            if (tags && p == 0) tags[slot] = tag;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(full + slot, ((has_f ? 9u : 0u) + (has_c ? 4u : 0u)) * segbytes);
        }
        __syncwarp();
        float* dst0 = stage + size_t(slot) * L.stage_elems();
        if (lane < 9 && has_f) {
            const int r = yf;
            const bool blo = walls && r == 0, bhi = walls && r == ny - 1;
            int pl = i, rr;
            if ((ey > 0 && blo) || (ey < 0 && bhi)) {
                pl = opp_of(i);
                rr = r;
            } else {
                rr = wrap_row(r - ey);
            }
            bulk_g2s(dst0 + size_t(lane) * segw, fs + size_t(pl) * P + size_t(rr) * pitch + x0,
                     segbytes, full + slot);
        } else if (lane >= 9 && lane < 13 && has_c) {
            const int rc = wrap_row(ycl);
            bulk_g2s(dst0 + size_t(lane) * segw,
                     cs + size_t(lane - 9) * P + size_t(rc) * pitch + x0, segbytes, full + slot);
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------- consumer
template <bool MRT, int S, int NWC = 0>
__device__ __forceinline__ void consume_tile_c(const DomDesc& D, int parity, int x0, int y0,
                                               int rows, unsigned char* __restrict__ smem, int nw,
                                               int cw, unsigned& q)
{
    const int NW = NWC > 0 ? NWC : nw;
    float* __restrict__ fd = static_cast<float*>(parity ? D.f[0] : D.f[1]);
    float* __restrict__ cd = static_cast<float*>(parity ? D.g[0] : D.g[1]);
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const int P = static_cast<int>(D.plane);
    const bool walls = D.walls != 0;
    const NodeParams<float> prm = node_params<float>(D);
    const StageLayoutC L(NW, S);
    const int segw = L.segw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    const float* stage = reinterpret_cast<const float*>(smem + L.stages());
    float* ering = reinterpret_cast<float*>(smem + L.erings()) + size_t(cw) * L.ering_elems();
    float* pring = reinterpret_cast<float*>(smem + L.prings()) + cw * 4 * 34;
    float* wring = reinterpret_cast<float*>(smem + L.wrings()) + cw * 34;  // new words of a row

    const int lane = threadIdx.x & 31;
    const TilePlanC T(y0, rows, ny, walls);
    const unsigned qb = q;
    q += unsigned(T.count());

    const int wx0 = x0 + 32 * cw;          // first column of this warp
    const int wcols = min(32, nx - wx0);   // may be <= 0 for a ragged tile
    const bool active = lane < wcols;
    const int ecols = wcols + 4;           // expanded columns: wx0-2 .. wx0+wcols+1
    const int x = wx0 + lane;
    const int ci = 32 * cw + lane + 4;     // segment index of the lane's column
    const int own = lane + 1;              // phi ring entry of the lane's column

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
    auto eslot = [&](int yl) -> float* {
        return ering + ((yl - y0 + 2) % kESlots) * (kEArrays * kECols);
    };
    auto rslot = [&](int y) -> float* { return pring + ((y - y0 + 1) & 3) * 34; };

    // 1. expand compact row yl (stage p): column j of the ring is lattice
    //    column wx0 - 2 + j, segment index 32 cw + j + 2
    auto expand = [&](int p, int yl) {
        const float* sc = stage_ptr(p) + 9 * segw;
        float* e = eslot(yl);
        for (int j = lane; j < ecols; j += 32) {
            const int si = 32 * cw + j + 2;
            const float word = sc[si];
            const float phi = G0<float>::value(word);
            float ge[9];
            g_equilibria<float>(phi, sc[segw + si], sc[2 * segw + si], sc[3 * segw + si], ge);
            e[j] = word;
#pragma unroll
            for (int a = 1; a < 9; ++a) e[a * kECols + j] = ge[a];
            e[9 * kECols + j] = g_tail_sum<float>(ge);
        }
    };
    // 2. phi(t+1) of real row r at ring column j; returns the new word
    auto phi_next = [&](int r, int j, float& phi_out) -> float {
        const bool blo = walls && r == 0, bhi = walls && r == ny - 1;
        const float* m = eslot(r);
        const float* b = blo ? m : eslot(r - 1);
        const float* a = bhi ? m : eslot(r + 1);
        const float g1 = m[1 * kECols + j - 1];
        const float g2 = m[2 * kECols + j + 1];
        const float g3 = blo ? m[4 * kECols + j] : b[3 * kECols + j];
        const float g4 = bhi ? m[3 * kECols + j] : a[4 * kECols + j];
        const float g5 = blo ? m[6 * kECols + j] : b[5 * kECols + j - 1];
        const float g6 = bhi ? m[5 * kECols + j] : a[6 * kECols + j + 1];
        const float g7 = blo ? m[8 * kECols + j] : b[7 * kECols + j + 1];
        const float g8 = bhi ? m[7 * kECols + j] : a[8 * kECols + j - 1];
        const float tail_in = (((g1 + g2) + (g3 + g4)) + ((g5 + g6) + (g7 + g8)));
        const float word = G0<float>::advance(m[j], tail_in - m[9 * kECols + j]);
        phi_out = G0<float>::value(word);
        return word;
    };
    // publish row r (real): phi(t+1) at the ring entries k = 0 .. wcols + 1
    // (lattice columns wx0 - 1 .. wx0 + wcols, expanded column j = k + 1),
    // every entry computed alike; the new words go to the word ring, from
    // which each lane takes its own (entry lane + 1) after a __syncwarp
    auto publish = [&](int r) {
        float* s = rslot(r);
        for (int k = lane; k < wcols + 2; k += 32) {
            float ph;
            wring[k] = phi_next(r, k + 1, ph);
            s[k] = ph;
        }
    };
    auto ghost_row = [&](int yg, int ys, float h2) {
        float* sg = rslot(yg);
        const float* ss = rslot(ys);
        for (int k = lane; k < wcols + 2; k += 32) sg[k] = ss[k] - h2;
    };
    // compact rows up to e expanded: is row r ready to publish?
    auto ready = [&](int r, int e) { return e >= min(r + 1, T.chi); };

    const int y1 = T.y1;
    const bool bottom_ghost = walls && y0 == 0;
    int pub = bottom_ghost ? 0 : y0 - 1;
    float wcur = 0.f, wnext = 0.f;
    int p = 0;
    // prologue: compact-only stages; publish rows y0-1 (unless a wall ghost) and y0
    for (; p < T.npro; ++p) {
        const int yl = T.clo + p;
        wait_full(p);
        if (wcols > 0) expand(p, yl);
        release(p);  // includes __syncwarp: the expanded row is visible to the warp
        while (pub <= y0 && ready(pub, yl)) {
            if (wcols > 0) publish(pub);
            __syncwarp();
            if (pub == y0 && active) wcur = wring[own];
            ++pub;
        }
        __syncwarp();  // publish reads the ring rows the next expansion overwrites
    }
    for (int y = y0; y < y1; ++y, ++p) {
        wait_full(p);
        if (wcols > 0 && y + 2 <= T.chi) expand(p, y + 2);
        __syncwarp();
        const int yn = y + 1;
        if (walls && yn == ny) {
            ghost_row(ny, ny - 2, 2.f * prm.h_top);
        } else if (wcols > 0) {
            publish(yn);
        }
        __syncwarp();
        if (!(walls && yn == ny) && active) wnext = wring[own];
        if (bottom_ghost && y == 0) ghost_row(-1, 1, 2.f * prm.h_bot);
        __syncwarp();
        if (active) {
            const bool blo = walls && y == 0, bhi = walls && y == ny - 1;
            const float* sb = stage_ptr(p);
            float f[9];
            read9<float>(sb, segw, ci, blo, bhi, f);
            const float* sm = rslot(y - 1);
            const float* sc = rslot(y);
            const float* sp = rslot(y + 1);
            const float c = sc[own];
            float dx, dy, lap;
            stencils<float>(c, sc[own + 1], sc[own - 1], sp[own], sm[own], sp[own + 1],
                            sp[own - 1], sm[own + 1], sm[own - 1], dx, dy, lap);
            const bool s2 = D.step2 && (blo || bhi);
            float fo[9], uxe, uye;
            collide_f<float, MRT>(prm, f, c, dx, dy, lap, s2, D.step2_relax_j != 0, fo, uxe, uye);
            const float G = gamma_mu<float>(prm, c, lap);
            const int o = y * pitch + x + kXOff;
            const float co[4] = {wcur, G, uxe, uye};
#pragma unroll
            for (int i = 0; i < 9; ++i) fd[i * P + o] = fo[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) cd[k * P + o] = co[k];
            // periodic ghost copies: logical 0, 1 also at nx, nx+1 and
            // logical nx-2, nx-1 also at -2, -1
            if (x < 2) {
#pragma unroll
                for (int i = 0; i < 9; ++i) fd[i * P + o + nx] = fo[i];
#pragma unroll
                for (int k = 0; k < 4; ++k) cd[k * P + o + nx] = co[k];
            }
            if (x >= nx - 2) {
#pragma unroll
                for (int i = 0; i < 9; ++i) fd[i * P + o - nx] = fo[i];
#pragma unroll
                for (int k = 0; k < 4; ++k) cd[k * P + o - nx] = co[k];
            }
        }
        release(p);
        wcur = wnext;
    }
}

}  // namespace lbfe
