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
// Pipeline.  A CTA of NW compute warps owns a strip of W = 64 NW - 4
// columns; each compute thread takes two adjacent columns in each of the
// three per-row phases below, so that each phase is one pass over the 32 NW
// compute threads (W + 4 expanded columns, W + 2 phi entries, W nodes) and
// most shared and global accesses move aligned pairs.  Warp 0 (the
// producer) copies, for stage p of a tile, the 9 pulled f segments of row y
// and the 4 compact segments of row y + 2 (rows above and below the tile
// get compact-only stages).  The compute threads then, per row,
//   1. expand the compact row they receive into the 8 outgoing g'_i, their
//      sum and the phi word, into a CTA-wide 3-row ring;
//   2. form phi(t+1) of row y + 1 from that ring into a CTA-wide 4-row phi
//      ring (and the new words into a 2-row word ring);
//   3. collide row y (f from the stage, the phi stencil from the ring, the
//      wall ghost rows mirrored on the fly) and store 9 f and 4 values.
// Phases 1 -> 2 and 2 -> 3 read what other warps wrote, so the compute warps
// meet twice per row at a named CTA barrier.  That barrier is a hardware
// wait, not a poll: every compute warp runs the same sequence of meetings
// whatever its bounded stage waits return, so it always completes.
#pragma once

#include "lb_async.cuh"
#include "lb_internal.h"
#include "lb_node.cuh"
#include "lb_node_x2.cuh"
#include "lb_step.cuh"

namespace lbfe {

constexpr int kStagesC = 2;    // stage-ring depth of the compact step
constexpr int kEArrays = 10;   // phi word, g'_1..g'_8, sum of g'_1..g'_8
constexpr int kESlots = 3;     // expanded rows kept
constexpr int kComputeBarrier = 1;  // named barrier of the compute warps

// Shared memory of one CTA (byte offsets): stage barriers (full at 0, empty
// at 64), S stages of 13 segments, the expanded-row ring, the phi ring and
// the word ring.  Every row of a ring and every segment starts on an 8-byte
// boundary (pairs) and is padded by 4 elements beyond the last pair read.
struct StageLayoutC {
    int NW, S, W, segw, EC, PC;
    __host__ __device__ StageLayoutC(int nw, int s)
        : NW(nw), S(s), W(compact_strip(32 * nw)), segw(64 * nw + 4), EC(64 * nw + 4),
          PC(64 * nw + 4)
    {
    }
    __host__ __device__ size_t full() const { return 0; }
    __host__ __device__ size_t empty() const { return 64; }
    __host__ __device__ size_t stages() const { return 128; }
    __host__ __device__ size_t stage_elems() const { return size_t(13) * segw; }
    __host__ __device__ size_t erings() const { return stages() + size_t(S) * stage_elems() * 4; }
    __host__ __device__ size_t ering_elems() const { return size_t(kESlots) * kEArrays * EC; }
    __host__ __device__ size_t prings() const { return erings() + ering_elems() * 4; }
    __host__ __device__ size_t wrings() const { return prings() + size_t(4) * PC * 4; }
    __host__ __device__ size_t total() const { return wrings() + size_t(2) * PC * 4; }
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

template <int S>
__device__ __forceinline__ void init_stages_c(unsigned char* smem, int NW)
{
    const StageLayoutC L(NW, S);
    if (threadIdx.x == 0) {
        uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
        uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
        for (int k = 0; k < S; ++k) {
            mbar_init(full + k, 1);
            mbar_init(empty + k, NW);
        }
        fence_mbar_init();
    }
    __syncthreads();
}

// ----------------------------------------------------------- producer
template <int S, int NWC = 0>
__device__ __forceinline__ void produce_tile_c(const DomDesc& D, int parity, int x0, int y0,
                                               int rows, int cols, unsigned char* __restrict__ smem,
                                               int nw, unsigned& q, int* tags = nullptr, int tag = 0)
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
    // columns x0-4 .. x0+ncols+3 (ncols rounded up to 4 keeps the copy a
    // multiple of 16 bytes), within the row's pitch
    const int ncols = cols > 0 ? cols : min(L.W, D.nx - x0);
    const int seglen = min(min(segw, (ncols + 3) / 4 * 4 + 8), pitch - x0);
    const uint32_t segbytes = uint32_t(seglen) * 4u;
    const int i = lane % 9;
    const int ey = ey_of(i);
    auto wrap_row = [&](int r) { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };
    for (int p = 0; p < T.count(); ++p, ++q) {
        const unsigned slot = q % unsigned(S);
        const unsigned use = q / unsigned(S);
        if (use > 0) mbar_wait_idle(empty + slot, (use - 1) & 1u, D.err);
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
// Pairs of consecutive elements in shared memory: an aligned pair (one
// 64-bit access) or any two (two 32-bit accesses).
__device__ __forceinline__ float2 ld_pair(const float* p)
{
    return *reinterpret_cast<const float2*>(p);
}
__device__ __forceinline__ float2 ld_two(const float* p) { return make_float2(p[0], p[1]); }
__device__ __forceinline__ void st_pair(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// Compute warp cw of NW; its thread t = 32 cw + lane handles expanded
// columns, phi entries and node columns j0 = 2t and j0 + 1 of the strip.
template <bool MRT, int S, int NWC = 0>
__device__ __forceinline__ void consume_tile_c(const DomDesc& D, int parity, int x0, int y0,
                                               int rows, int cols, unsigned char* __restrict__ smem,
                                               int nw, int cw, unsigned& q)
{
    const int NW = NWC > 0 ? NWC : nw;
    float* __restrict__ fd = static_cast<float*>(parity ? D.f[0] : D.f[1]);
    float* __restrict__ cd = static_cast<float*>(parity ? D.g[0] : D.g[1]);
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const int P = static_cast<int>(D.plane);
    const bool walls = D.walls != 0;
    const NodeParams<float> prm = node_params<float>(D);
    const StageLayoutC L(NW, S);
    const int segw = L.segw, EC = L.EC, PC = L.PC;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    const float* stage = reinterpret_cast<const float*>(smem + L.stages());
    float* ering = reinterpret_cast<float*>(smem + L.erings());
    float* pring = reinterpret_cast<float*>(smem + L.prings());
    float* wring = reinterpret_cast<float*>(smem + L.wrings());

    const int lane = threadIdx.x & 31;
    const int j0 = 2 * (32 * cw + lane);
    const TilePlanC T(y0, rows, ny, walls);
    const unsigned qb = q;
    q += unsigned(T.count());

    const int ncols = cols > 0 ? cols : min(L.W, nx - x0);  // node columns of this strip
    // a thread works on its pair when the first column of it is in use (the
    // second one, if not, is computed from stale data and never stored)
    const bool e_on = j0 < ncols + 4;  // expanded column j: lattice x0 - 2 + j
    const bool p_on = j0 < ncols + 2;  // phi entry k: lattice x0 - 1 + k
    const bool n_on = j0 < ncols;      // node column n: lattice x0 + n
    const int x = x0 + j0;

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
    // all compute warps meet: writes before the meeting are visible to reads
    // after it
    auto meet = [&]() {
        __syncwarp();
        named_sync(kComputeBarrier, 32 * NW);
    };
    auto eslot = [&](int yl) -> float* {
        return ering + ((yl - y0 + 2) % kESlots) * (kEArrays * EC);
    };
    auto rslot = [&](int y) -> float* { return pring + ((y - y0 + 1) & 3) * PC; };
    auto wslot = [&](int y) -> float* { return wring + (y & 1) * PC; };

    // 1. expand compact row yl (stage p): columns j0, j0 + 1 (segment
    //    indices j0 + 2, j0 + 3)
    auto expand = [&](int p, int yl) {
        if (!e_on) return;
        const float* sc = stage_ptr(p) + 9 * segw + j0 + 2;
        float* e = eslot(yl) + j0;
        const f2 w2 = ld_pair(sc);
        f2 ge[9];
        g_equilibria2(g0_value2(w2), ld_pair(sc + segw), ld_pair(sc + 2 * segw),
                      ld_pair(sc + 3 * segw), ge);
        st_pair(e, w2.v);
#pragma unroll
        for (int a = 1; a < 9; ++a) st_pair(e + a * EC, ge[a].v);
        st_pair(e + 9 * EC, g_tail_sum2(ge).v);
    };
    // 2. phi(t+1) of real row r at entries j0, j0 + 1 (expanded columns
    //    j0 + 1, j0 + 2); g'_i arrives from expanded column j - e_x of row
    //    r - e_y, or, through a wall, as g'_opp(i) of the node itself
    auto publish = [&](int r) {
        if (!p_on) return;
        const bool blo = walls && r == 0, bhi = walls && r == ny - 1;
        const float* m = eslot(r) + j0;
        const f2 g1 = ld_pair(m + 1 * EC), g2 = ld_pair(m + 2 * EC + 2);
        f2 g3, g4, g5, g6, g7, g8;
        if (blo) {
            g3 = ld_two(m + 4 * EC + 1);
            g5 = ld_two(m + 6 * EC + 1);
            g7 = ld_two(m + 8 * EC + 1);
        } else {
            const float* b = eslot(r - 1) + j0;
            g3 = ld_two(b + 3 * EC + 1);
            g5 = ld_pair(b + 5 * EC);
            g7 = ld_pair(b + 7 * EC + 2);
        }
        if (bhi) {
            g4 = ld_two(m + 3 * EC + 1);
            g6 = ld_two(m + 5 * EC + 1);
            g8 = ld_two(m + 7 * EC + 1);
        } else {
            const float* a = eslot(r + 1) + j0;
            g4 = ld_two(a + 4 * EC + 1);
            g6 = ld_pair(a + 6 * EC + 2);
            g8 = ld_pair(a + 8 * EC);
        }
        const f2 tail_in = (((g1 + g2) + (g3 + g4)) + ((g5 + g6) + (g7 + g8)));
        const f2 word = g0_advance2(f2(ld_two(m + 1)), tail_in - f2(ld_two(m + 9 * EC + 1)));
        st_pair(rslot(r) + j0, g0_value2(word).v);
        st_pair(wslot(r) + j0, word.v);
    };
    // compact rows up to e expanded: is row r ready to publish?
    auto ready = [&](int r, int e) { return e >= min(r + 1, T.chi); };

    const int y1 = T.y1;
    int pub = (walls && y0 == 0) ? 0 : y0 - 1;
    int p = 0;
    // prologue: compact-only stages; publish rows y0-1 (unless a wall ghost) and y0
    for (; p < T.npro; ++p) {
        const int yl = T.clo + p;
        wait_full(p);
        expand(p, yl);
        release(p);
        meet();
        bool any = false;
        while (pub <= y0 && ready(pub, yl)) {
            publish(pub);
            ++pub;
            any = true;
        }
        if (any) meet();
    }
    const float h2b = 2.f * prm.h_bot, h2t = 2.f * prm.h_top;
    for (int y = y0; y < y1; ++y, ++p) {
        wait_full(p);
        if (y + 2 <= T.chi) expand(p, y + 2);
        meet();
        const int yn = y + 1;
        if (!(walls && yn == ny)) publish(yn);
        meet();
        if (n_on) {
            const bool blo = walls && y == 0, bhi = walls && y == ny - 1;
            // pulled f of nodes j0, j0 + 1 (segment indices j0 + 4, j0 + 5);
            // through a wall the stage holds the node's own f_opp(i)
            const float* sb = stage_ptr(p) + j0 + 4;
            float2 f2x[9];
            f2x[0] = ld_pair(sb);
            f2x[1] = ld_two(sb + segw - 1);
            f2x[2] = ld_two(sb + 2 * segw + 1);
            f2x[3] = ld_pair(sb + 3 * segw);
            f2x[4] = ld_pair(sb + 4 * segw);
            f2x[5] = blo ? ld_pair(sb + 5 * segw) : ld_two(sb + 5 * segw - 1);
            f2x[6] = bhi ? ld_pair(sb + 6 * segw) : ld_two(sb + 6 * segw + 1);
            f2x[7] = blo ? ld_pair(sb + 7 * segw) : ld_two(sb + 7 * segw + 1);
            f2x[8] = bhi ? ld_pair(sb + 8 * segw) : ld_two(sb + 8 * segw - 1);
            // phi entries j0 .. j0 + 3 of rows y - 1, y, y + 1 (centres j0 + 1,
            // j0 + 2); the wall ghost rows are mirrors of rows 1 and ny - 2
            const float* rc = rslot(y) + j0;
            const float2 c01 = ld_pair(rc), c23 = ld_pair(rc + 2);
            float2 n01, n23, s01, s23;
            if (bhi) {
                const float* rq = rslot(ny - 2) + j0;
                const float2 a01 = ld_pair(rq), a23 = ld_pair(rq + 2);
                n01 = make_float2(a01.x - h2t, a01.y - h2t);
                n23 = make_float2(a23.x - h2t, a23.y - h2t);
            } else {
                const float* rq = rslot(y + 1) + j0;
                n01 = ld_pair(rq);
                n23 = ld_pair(rq + 2);
            }
            if (blo) {
                const float* rq = rslot(1) + j0;
                const float2 a01 = ld_pair(rq), a23 = ld_pair(rq + 2);
                s01 = make_float2(a01.x - h2b, a01.y - h2b);
                s23 = make_float2(a23.x - h2b, a23.y - h2b);
            } else {
                const float* rq = rslot(y - 1) + j0;
                s01 = ld_pair(rq);
                s23 = ld_pair(rq + 2);
            }
            const bool s2 = D.step2 && (blo || bhi);
            // centres (j0 + 1, j0 + 2), east (j0 + 2, j0 + 3), west (j0, j0 + 1)
            const f2 c(c01.y, c23.x);
            f2 dx, dy, lap;
            stencils2(c, c23, c01, f2(n01.y, n23.x), f2(s01.y, s23.x), n23, n01, s23, s01, dx, dy,
                      lap);
            f2 fi[9], fo2[9], uxe, uye;
#pragma unroll
            for (int i = 0; i < 9; ++i) fi[i] = f2x[i];
            collide_f2<MRT>(prm, fi, c, dx, dy, lap, s2, D.step2_relax_j != 0, fo2, uxe, uye);
            const f2 co2[4] = {f2(ld_two(wslot(y) + j0 + 1)), gamma_mu2(prm, c, lap), uxe, uye};
            float fo[2][9], co[2][4];
#pragma unroll
            for (int l = 0; l < 2; ++l) {
#pragma unroll
                for (int i = 0; i < 9; ++i) fo[l][i] = fo2[i].lane(l);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) co[l][kk] = co2[kk].lane(l);
            }
            const int o = y * pitch + x + kXOff;  // even: pairs are 8-byte aligned
            if (j0 + 1 < ncols) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    *reinterpret_cast<float2*>(fd + i * P + o) = make_float2(fo[0][i], fo[1][i]);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    *reinterpret_cast<float2*>(cd + kk * P + o) = make_float2(co[0][kk], co[1][kk]);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) fd[i * P + o] = fo[0][i];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) cd[kk * P + o] = co[0][kk];
            }
            // periodic ghost copies: logical 0, 1 also at nx, nx+1 and
            // logical nx-2, nx-1 also at -2, -1
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const int xl = x + l;
                if (j0 + l >= ncols) continue;
                if (xl < 2) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fd[i * P + o + l + nx] = fo[l][i];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) cd[kk * P + o + l + nx] = co[l][kk];
                }
                if (xl >= nx - 2) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fd[i * P + o + l - nx] = fo[l][i];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) cd[kk * P + o + l - nx] = co[l][kk];
                }
            }
        }
        release(p);
    }
}

}  // namespace lbfe
