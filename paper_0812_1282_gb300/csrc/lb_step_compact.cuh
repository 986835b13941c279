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
// Pipeline.  A CTA has a producer warp and NW compute warps.  For stage p
// of a tile the producer copies the 4 compact segments of row q = clo + p
// and, once the tile's rows start, the 9 pulled f segments of row q - 3.
// In the iteration of stage p every compute warp, with no help from the
// others:
//   1. expands compact row q over 64 columns (two per thread) into the 8
//      outgoing g'_i of each column, in registers;
//   2. hands the values that leave a column sideways to its neighbours with
//      warp shuffles and sums what each column receives by source row:
//        U(q+1) = g'_3 + g'_5 + g'_7 from row q (moving up),
//        H(q)   = g'_1 + g'_2 from row q,
//        D(q-1) = g'_4 + g'_6 + g'_8 from row q (moving down),
//      (through a wall the node's own opposite populations stand in);
//   3. forms phi(t+1) of row q - 1 = U + H + D, whose U and H it kept from
//      the two previous iterations, into a CTA-wide 4-row phi ring (and the
//      new words into a 4-row word ring).
// Warp w expands the columns 62 w .. 62 w + 63 of the strip: consecutive
// warps overlap by two columns, so every column's three sums are complete
// in one warp (its first and last column in the other).  In the same
// iteration each compute warp
//   4. collides row q - 3 (f from the stage, the phi stencil of rows q - 4
//      .. q - 2 from the ring, the wall ghost rows mirrored on the fly; two
//      nodes per thread) and stores 9 f and 4 values.
// Steps 1-3 and step 4 touch different rows, so a warp can overlap them;
// the compute warps meet once per iteration, at a named CTA barrier, after
// which the phi of row q - 1 is visible to every warp.
// The strip has W = 62 NW - 2 node columns, rounded down to a multiple of 4.
// The barrier is a hardware wait, not a poll: every compute warp runs the
// same sequence of meetings whatever its bounded stage waits return, so it
// always completes.
#pragma once

#include "lb_async.cuh"
#include "lb_internal.h"
#include "lb_node.cuh"
#include "lb_node_x2.cuh"
#include "lb_step.cuh"

namespace lbfe {

constexpr int kStagesC = 3;          // stage-ring depth of the compact step
constexpr int kComputeBarrier = 1;   // named barrier of the compute warps

// Shared memory of one CTA (byte offsets): stage barriers (full at 0, empty
// at 64), S stages of 13 segments, the phi ring and the word ring.  Every
// segment and ring row starts on a 16-byte boundary and holds 64 NW + 4
// elements, beyond the last pair any thread reads.
struct StageLayoutC {
    int NW, S, W, segw, PC;
    __host__ __device__ StageLayoutC(int nw, int s)
        : NW(nw), S(s), W(compact_strip(32 * nw)), segw(64 * nw + 4), PC(64 * nw + 4)
    {
    }
    __host__ __device__ size_t full() const { return 0; }
    __host__ __device__ size_t empty() const { return 64; }
    __host__ __device__ size_t stages() const { return 128; }
    __host__ __device__ size_t stage_elems() const { return size_t(13) * segw; }
    __host__ __device__ size_t prings() const { return stages() + size_t(S) * stage_elems() * 4; }
    __host__ __device__ size_t wrings() const { return prings() + size_t(4) * PC * 4; }
    __host__ __device__ size_t total() const { return wrings() + size_t(4) * PC * 4; }
};

// Stages of one tile: stage p carries the compact row q = clo + p when
// q <= chi, and from p = npro on (q = y + 3 for tile row y) the f of row y.
// clo = y0 - 2 and chi = y1 + 1, clipped to the lattice with walls; every
// stage up to the tile's last row exists even where it carries nothing, so
// that q runs without gaps.  Rows are logical (not wrapped).
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
        npro = y0 + 3 - clo;
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
        const int yf = p < T.npro ? -1 : y0 + (p - T.npro);  // f row (or none)
        const int ycl = T.clo + p;                            // compact row (logical)
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

// Compute warp cw of NW.  Its lane expands columns je, je + 1 (je = 62 cw +
// 2 lane; strip column j is lattice column x0 - 2 + j) and collides nodes
// jn, jn + 1 (jn = 2 (32 cw + lane); node n is lattice column x0 + n).  The
// phi and word rings are indexed by strip column j.  With PRM_SMEM the node
// parameters (and the wall wetting gradients) come from prm_shared, a copy
// in shared memory read at each use, instead of registers held for the
// whole tile (the batched form, whose parameters change from tile to tile).
// seal: a whole-domain strip completes the edge sectors of its rows (below).
template <bool MRT, int S, int NWC = 0, bool PRM_SMEM = false>
__device__ __forceinline__ void consume_tile_c(const DomDesc& D, int parity, int x0, int y0,
                                               int rows, int cols, unsigned char* __restrict__ smem,
                                               int nw, int cw, unsigned& q,
                                               const NodeParams<float>* prm_shared = nullptr,
                                               bool seal = false)
{
    const int NW = NWC > 0 ? NWC : nw;
    float* __restrict__ fd = static_cast<float*>(parity ? D.f[0] : D.f[1]);
    float* __restrict__ cd = static_cast<float*>(parity ? D.g[0] : D.g[1]);
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const int P = static_cast<int>(D.plane);
    const bool walls = D.walls != 0;
    const NodeParams<float> prm = node_params<float>(D);
    const StageLayoutC L(NW, S);
    const int segw = L.segw, PC = L.PC;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.full());
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + L.empty());
    const float* stage = reinterpret_cast<const float*>(smem + L.stages());
    float* pring = reinterpret_cast<float*>(smem + L.prings());
    float* wring = reinterpret_cast<float*>(smem + L.wrings());

    const int lane = threadIdx.x & 31;
    const int je = 62 * cw + 2 * lane;
    const int jn = 2 * (32 * cw + lane);
    const TilePlanC T(y0, rows, ny, walls);
    const unsigned qb = q;
    q += unsigned(T.count());

    const int ncols = cols > 0 ? cols : min(L.W, nx - x0);  // node columns of this strip
    const bool n_on = jn < ncols;
    const int x = x0 + jn;
    // A strip that covers its whole domain takes the periodic wrap from its
    // own stage copy: lattice column c < 0 or c >= nx is read at stage
    // index (c mod nx) + 4 instead of the ghost columns, whose copies such a
    // strip therefore neither uses nor keeps.  Only the few lanes whose columns
    // wrap do anything extra.  Expansion lane: columns je - 2, je - 1 of the
    // domain (stage indices ex0, ex1); collision lane: pulls across x = 0 or
    // x = nx - 1.
    // One bit mask keeps the lane's wrap cases (the indices are recomputed
    // on the rare path): 1 expansion columns wrap, 2 node jn pulls from
    // x = -1, 4 node jn pulls from x = nx, 8 node jn + 1 pulls from x = nx;
    // 16 marks a whole strip, 32 one that seals its rows' edge sectors.
    const bool whole = x0 == 0 && ncols == nx;
    auto wrap_idx = [nx](int c) { return (c < 0 ? c + nx : (c >= nx ? c - nx : c)) + 4; };
    const unsigned wrapbits =
        whole ? (unsigned(wrap_idx(je - 2) != je + 2 || wrap_idx(je - 1) != je + 3) |
                 (unsigned(jn == 0) << 1) | (unsigned(jn + 1 == nx) << 2) |
                 (unsigned(jn + 2 == nx) << 3) | 16u | (seal ? 32u : 0u))
              : 0u;

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
    // consecutive rows take the four ring rows in turn; an iteration touches
    // four consecutive rows (it reads q - 4 .. q - 2 and writes q - 1)
    auto rslot = [&](int y) -> float* { return pring + ((y - y0 + 1) & 3) * PC; };
    auto wslot = [&](int y) -> float* { return wring + ((y - y0 + 1) & 3) * PC; };

    // real rows whose phi(t+1) the tile needs (wall ghost rows are mirrors)
    const int pub_lo = (walls && y0 == 0) ? 0 : y0 - 1;
    const int pub_hi = walls ? min(T.y1, ny - 1) : T.y1;
    // the sums of rows q and q - 1 carried from iteration to iteration
    const f2 zero(0.f);
    f2 u_next = zero;                 // U(q + 1)
    f2 uh = zero, wd = zero, tl = zero;  // U + H, phi word, tail of row q - 1
    f2 d_wall = zero;                 // D of the top wall row, from that row itself
    const unsigned kAll = 0xffffffffu;
    for (int p = 0; p < T.count(); ++p) {
        const int qr = T.clo + p;  // compact row of this stage
        wait_full(p);
        f2 d_pub = d_wall;         // D of row qr - 1
        f2 uh_q = zero, wd_q = zero, tl_q = zero;
        const bool has_c = qr <= T.chi;
        if (has_c) {
            // 1. expand (every lane: all take part in the shuffles)
            const float* sc = stage_ptr(p) + 9 * segw + je + 2;
            float2 cv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) cv[k] = ld_pair(sc + k * segw);
            if (wrapbits & 1u) {
                const float* sw = stage_ptr(p) + 9 * segw;
                const int ex0 = wrap_idx(je - 2), ex1 = wrap_idx(je - 1);
#pragma unroll
                for (int k = 0; k < 4; ++k) cv[k] = make_float2(sw[k * segw + ex0], sw[k * segw + ex1]);
            }
            wd_q = f2(cv[0]);
            f2 ge[9];
            g_equilibria2(g0_value2(wd_q), f2(cv[1]), f2(cv[2]), f2(cv[3]), ge);
            tl_q = g_tail_sum2(ge);
            // 2. what enters column je from the left and je + 1 from the right
            const f2 g5l(__shfl_up_sync(kAll, ge[5].v.y, 1), ge[5].v.x);
            const f2 g1l(__shfl_up_sync(kAll, ge[1].v.y, 1), ge[1].v.x);
            const f2 g8l(__shfl_up_sync(kAll, ge[8].v.y, 1), ge[8].v.x);
            const f2 g7r(ge[7].v.y, __shfl_down_sync(kAll, ge[7].v.x, 1));
            const f2 g2r(ge[2].v.y, __shfl_down_sync(kAll, ge[2].v.x, 1));
            const f2 g6r(ge[6].v.y, __shfl_down_sync(kAll, ge[6].v.x, 1));
            const f2 h_q = g1l + g2r;
            const f2 u_q = (walls && qr == 0) ? (ge[4] + ge[6]) + ge[8] : u_next;
            uh_q = u_q + h_q;
            d_pub = (ge[4] + g6r) + g8l;
            u_next = (ge[3] + g5l) + g7r;
            if (walls && qr == ny - 1) d_wall = (ge[3] + ge[5]) + ge[7];
        }
        // 3. phi(t+1) of row qr - 1
        const int r = qr - 1;
        if (r >= pub_lo && r <= pub_hi) {
            const f2 word = g0_advance2(wd, (uh + d_pub) - tl);
            const f2 phi = g0_value2(word);
            float* pr = rslot(r) + je;
            float* wr = wslot(r) + je;
            // a warp's first and last column are complete in its neighbours
            if (lane > 0 && lane < 31) {
                st_pair(pr, phi.v);
                st_pair(wr, word.v);
            } else if (lane == 0) {
                pr[1] = phi.v.y;
                wr[1] = word.v.y;
            } else {
                pr[0] = phi.v.x;
                wr[0] = word.v.x;
            }
        }
        uh = uh_q;
        wd = wd_q;
        tl = tl_q;
        // 4. collide row y = qr - 3 (rows q - 4 .. q - 2 of the ring were
        //    published before the previous meeting)
        const int y = qr - 3;
        if (p >= T.npro && n_on) {
            const bool blo = walls && y == 0, bhi = walls && y == ny - 1;
            // pulled f of nodes jn, jn + 1 (segment indices jn + 4, jn + 5);
            // through a wall the stage holds the node's own f_opp(i)
            const float* sb = stage_ptr(p) + jn + 4;
            f2 fi[9];
            fi[0] = ld_pair(sb);
            fi[1] = ld_two(sb + segw - 1);
            fi[2] = ld_two(sb + 2 * segw + 1);
            fi[3] = ld_pair(sb + 3 * segw);
            fi[4] = ld_pair(sb + 4 * segw);
            fi[5] = blo ? ld_pair(sb + 5 * segw) : ld_two(sb + 5 * segw - 1);
            fi[6] = bhi ? ld_pair(sb + 6 * segw) : ld_two(sb + 6 * segw + 1);
            fi[7] = blo ? ld_pair(sb + 7 * segw) : ld_two(sb + 7 * segw + 1);
            fi[8] = bhi ? ld_pair(sb + 8 * segw) : ld_two(sb + 8 * segw - 1);
            if (wrapbits & 14u) {
                // whole-domain strip: pulls across the periodic boundary read
                // the stage copy at the wrapped column (stage index nx + 3 for
                // x = -1, 4 for x = nx)
                const float* st = stage_ptr(p);
                if (wrapbits & 2u) {
                    fi[1].v.x = st[segw + nx + 3];
                    if (!blo) fi[5].v.x = st[5 * segw + nx + 3];
                    if (!bhi) fi[8].v.x = st[8 * segw + nx + 3];
                }
                if (wrapbits & 4u) {
                    fi[2].v.x = st[2 * segw + 4];
                    if (!bhi) fi[6].v.x = st[6 * segw + 4];
                    if (!blo) fi[7].v.x = st[7 * segw + 4];
                }
                if (wrapbits & 8u) {
                    fi[2].v.y = st[2 * segw + 4];
                    if (!bhi) fi[6].v.y = st[6 * segw + 4];
                    if (!blo) fi[7].v.y = st[7 * segw + 4];
                }
            }
            // phi of strip columns jn + 1 .. jn + 4 of rows y - 1, y, y + 1
            // (centres jn + 2, jn + 3); a wall ghost row is row k - 1 (or
            // ny - k) less k h: the mirror (k = 2) or one-sided (k = 1) rule
            auto row3 = [&](const float* rw, f2& w, f2& c, f2& e) {
                const float2 a = ld_pair(rw + jn), b = ld_pair(rw + jn + 2),
                             d = ld_pair(rw + jn + 4);
                w = f2(a.y, b.x);
                c = f2(b);
                e = f2(b.y, d.x);
            };
            f2 cw_, cc, ce, nw_, nc, ne, sw, sc_, se;
            row3(rslot(y), cw_, cc, ce);
            if (bhi) {
                row3(rslot(ny - D.wet_k), nw_, nc, ne);
                const f2 h(float(D.wet_k) * (PRM_SMEM ? prm_shared->h_top : prm.h_top));
                nw_ = nw_ - h;
                nc = nc - h;
                ne = ne - h;
            } else {
                row3(rslot(y + 1), nw_, nc, ne);
            }
            if (blo) {
                row3(rslot(D.wet_k - 1), sw, sc_, se);
                const f2 h(float(D.wet_k) * (PRM_SMEM ? prm_shared->h_bot : prm.h_bot));
                sw = sw - h;
                sc_ = sc_ - h;
                se = se - h;
            } else {
                row3(rslot(y - 1), sw, sc_, se);
            }
            f2 dx, dy, lap;
            stencils2(cc, ce, cw_, nc, sc_, ne, nw_, se, sw, dx, dy, lap);
            const bool s2 = D.step2 && (blo || bhi);
            f2 fo2[9], uxe, uye, gmu;
            if constexpr (PRM_SMEM) {
                const volatile NodeParams<float>& PV = *prm_shared;
                collide_f2<MRT>(PV, fi, cc, dx, dy, lap, s2, D.step2_relax_j != 0, fo2, uxe, uye);
                gmu = gamma_mu2(PV, cc, lap);
            } else {
                collide_f2<MRT>(prm, fi, cc, dx, dy, lap, s2, D.step2_relax_j != 0, fo2, uxe, uye);
                gmu = gamma_mu2(prm, cc, lap);
            }
            const f2 co2[4] = {f2(ld_pair(wslot(y) + jn + 2)), gmu, uxe, uye};
            const int o = y * pitch + x + kXOff;  // even: pairs are 8-byte aligned
            if (jn + 1 < ncols) {
#pragma unroll
                for (int i = 0; i < 9; ++i) *reinterpret_cast<float2*>(fd + i * P + o) = fo2[i].v;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) *reinterpret_cast<float2*>(cd + kk * P + o) = co2[kk].v;
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) fd[i * P + o] = fo2[i].v.x;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) cd[kk * P + o] = co2[kk].v.x;
            }
            // periodic ghost copies: logical 0, 1 also at nx, nx+1 and
            // logical nx-2, nx-1 also at -2, -1 (a whole-domain strip wraps
            // in its stage copy instead)
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                if (wrapbits & 16u) break;
                const int xl = x + l;
                if (jn + l >= ncols) continue;
                if (xl < 2) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fd[i * P + o + l + nx] = fo2[i].lane(l);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) cd[kk * P + o + l + nx] = co2[kk].lane(l);
                }
                if (xl >= nx - 2) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fd[i * P + o + l - nx] = fo2[i].lane(l);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) cd[kk * P + o + l - nx] = co2[kk].lane(l);
                }
            }
        }
        // Sealing: a whole strip's node stores alone write the first and
        // last 32-byte sector of each output row in part, and a partly
        // written sector costs the memory a read before its write; so lanes
        // 0..12 of warp 0 zero physical columns 0..3 of plane `lane` (slack
        // and the ghost copies, stale in such a strip) and lanes 16..28 the
        // columns past the last node up to the sector end.  It pays where
        // the memory is the bound (many narrow domains in full use) and
        // costs warp 0 some twenty instructions per row where latency is.
        if ((wrapbits & 32u) && cw == 0 && p >= T.npro && (lane < 13 || (lane >= 16 && lane < 29))) {
            const int pl = lane < 13 ? lane : lane - 16;
            float* row = (pl < 9 ? fd + pl * P : cd + (pl - 9) * P) + (qr - 3) * pitch;
            if (lane < 13) {
                *reinterpret_cast<float4*>(row) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const int e = D.nx + kXOff;
                for (int k = e; k < ((e + 7) & ~7); ++k) row[k] = 0.f;
            }
        }
        release(p);
        meet();
    }
}

}  // namespace lbfe
