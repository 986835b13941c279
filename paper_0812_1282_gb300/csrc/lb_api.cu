// Host implementation of the C ABI declared in include/lbfe.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <unordered_map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbfe.h"
#include "lb_internal.h"
#include "lb_geo_persist.h"
#include "lb_node.cuh"

using lbfe::DomDesc;
using lbfe::StatsOut;
using lbfe::WorkItem;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define LB_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(LB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kMinBlockX = 32;
constexpr int kMaxBlockX = 256;
constexpr int kMaxBlockXCompact = 288;
constexpr int kGraphBig = 64;
// Items a work item of a persistent schedule may wait for: its own and the
// two neighbouring row blocks on each side (a short last block can bring
// the second one within reach), each in its own and the two neighbouring
// strips.
constexpr int kMaxDeps = 15;
constexpr int kGraphSmall = 2;
constexpr int kChunk = 1 << 20;  // nodes per staging chunk for host field output

// rest-state weights of f (deviation storage): t_0 = 4/9, t_1..4 = 1/9, t_5..8 = 1/36
const double kRest[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                         1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Row pitch in elements: nx logical columns, kXOff leading columns (two of
// them periodic ghosts), two trailing ghosts and slack; 128-byte multiple.
int pitch_for(int nx, int precision)
{
    const int per128 = precision == LB_FP32 ? 32 : 16;  // elements per 128 bytes
    return (nx + 8 + per128 - 1) / per128 * per128;
}

// Layout of a handle's device memory.
struct Layout {
    std::vector<size_t> dom_off;  // offset of domain d's buffer 0 (buffer 1 follows)
    std::vector<size_t> dom_bytes;  // bytes of one ping-pong buffer of domain d
    std::vector<size_t> geo_off;    // domain d's obstacle map (nx*ny bytes)
    std::vector<size_t> geo_flags;  // its persistent step's tile flags and counter (ints)
    size_t flags = 0, dep_off = 0, dep_idx = 0;  // persistent schedules (batches)
    size_t descs = 0, items = 0, partials = 0, stats = 0, pts = 0, count = 0, staging = 0, err = 0,
           sched = 0;
    size_t total = 0;
    long long item_cap = 0;
    int pts_cap = 0;
    long long staging_nodes = 0;
};

bool build_layout(int precision, int n_dom, const int* nx, const int* ny, Layout& L)
{
    if (n_dom < 1 || !nx || !ny) return false;
    const size_t es = precision == LB_FP32 ? 4 : 8;
    size_t off = 0;
    long long max_nodes = 0, item_cap = 0, max_nx = 0;
    int pts_cap = 0;
    for (int d = 0; d < n_dom; ++d) {
        if (nx[d] < 3 || ny[d] < 3) return false;
        const long long plane = (long long)pitch_for(nx[d], precision) * ny[d];
        if (9 * plane >= (1LL << 31)) return false;
        const size_t buf = align_up(size_t(18) * size_t(plane) * es, kAlign);
        L.dom_off.push_back(off);
        L.dom_bytes.push_back(buf);
        off += 2 * buf;
        // room for an obstacle map
        const size_t nodes = size_t(nx[d]) * size_t(ny[d]);
        L.geo_off.push_back(off);
        off = align_up(off + nodes, kAlign);
        L.geo_flags.push_back(off);
        off = align_up(off + sizeof(int) * (size_t(lbfe::geo_tiles(nx[d], ny[d])) + 1), kAlign);
        max_nodes = std::max(max_nodes, (long long)nx[d] * ny[d]);
        max_nx = std::max<long long>(max_nx, nx[d]);
        // at most ceil(nx / 28) strips per row (the narrowest strip of any
        // step is wider) and one tile row per lattice row
        item_cap += (long long)((nx[d] + 27) / 28) * ny[d];
        pts_cap = std::max(pts_cap, 16 * (nx[d] + ny[d]));
    }
    L.item_cap = item_cap;
    L.pts_cap = pts_cap;
    // at least one full row, so host field output can always go row by row
    L.staging_nodes = std::max(std::min<long long>(max_nodes, kChunk), max_nx);
    L.descs = off;
    off = align_up(off + sizeof(DomDesc) * n_dom, kAlign);
    L.items = off;
    off = align_up(off + sizeof(WorkItem) * (n_dom > 1 ? item_cap : 1), kAlign);
    L.flags = off;
    off = align_up(off + sizeof(int) * (n_dom > 1 ? item_cap : 1), kAlign);
    L.dep_off = off;
    off = align_up(off + sizeof(int) * (n_dom > 1 ? item_cap + 1 : 1), kAlign);
    L.dep_idx = off;
    off = align_up(off + sizeof(int) * (n_dom > 1 ? item_cap * kMaxDeps : 1), kAlign);
    L.partials = off;
    off = align_up(off + sizeof(double) * lbfe::kStatsFields * lbfe::max_partials_needed(0, 0),
                   kAlign);
    L.stats = off;
    off = align_up(off + sizeof(StatsOut), kAlign);
    L.pts = off;
    off = align_up(off + sizeof(double) * 2 * pts_cap, kAlign);
    L.count = off;
    off = align_up(off + sizeof(int), kAlign);
    L.err = off;
    off = align_up(off + sizeof(unsigned), kAlign);
    L.sched = off;
    off = align_up(off + 2 * sizeof(int) * LB_MAX_SCHED_CLASSES, kAlign);
    L.staging = off;
    off = align_up(off + sizeof(double) * 4 * L.staging_nodes, kAlign);
    L.total = off;
    return true;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int validate(const lb_params* p)
{
    if (!p) return fail(LB_ERR_INVALID_ARG, "params is NULL");
    if (!finite_pos(p->a) || !finite_pos(p->kappa) || !finite_pos(p->gamma_mob))
        return fail(LB_ERR_INVALID_ARG, "a, kappa and gamma_mob must be finite and > 0");
    if (!std::isfinite(p->tau_phi) || p->tau_phi <= 0.5)
        return fail(LB_ERR_INVALID_ARG, "tau_phi must be > 1/2");
    if (!std::isfinite(p->tau_alpha) || !std::isfinite(p->tau_beta))
        return fail(LB_ERR_INVALID_ARG, "tau_alpha / tau_beta must be finite");
    for (double ph : {-1.1, 1.1}) {
        const double tau = p->tau_beta + 0.5 * (ph + 1.0) * (p->tau_alpha - p->tau_beta);
        if (tau <= 0.5)
            return fail(LB_ERR_INVALID_ARG, "tau_rho(phi=%g) = %g <= 1/2", ph, tau);
    }
    if (!std::isfinite(p->h_bottom) || !std::isfinite(p->h_top))
        return fail(LB_ERR_INVALID_ARG, "wetting gradients must be finite");
    if (p->collision != LB_BGK && p->collision != LB_MRT)
        return fail(LB_ERR_INVALID_ARG, "collision must be LB_BGK or LB_MRT");
    if (p->precision != LB_FP32 && p->precision != LB_FP64)
        return fail(LB_ERR_INVALID_ARG, "precision must be LB_FP32 or LB_FP64");
    if (p->walls != 0 && p->walls != 1) return fail(LB_ERR_INVALID_ARG, "walls must be 0 or 1");
    if (p->step2_relax_momentum != 0 && p->step2_relax_momentum != 1)
        return fail(LB_ERR_INVALID_ARG, "step2_relax_momentum must be 0 or 1");
    if (p->mrt_lut != 0 && (p->mrt_lut < 2 || p->mrt_lut > (1 << 24) || p->collision != LB_MRT))
        return fail(LB_ERR_INVALID_ARG, "mrt_lut must be 0, or 2..2^24 with LB_MRT");
    if (p->compact_g != 0 && p->compact_g != 1)
        return fail(LB_ERR_INVALID_ARG, "compact_g must be 0 or 1");
    if (p->compact_g && (p->precision != LB_FP32 || p->tau_phi != 1.0))
        return fail(LB_ERR_INVALID_ARG, "compact_g needs LB_FP32 and tau_phi = 1");
    if (p->wetting_rule != 0 && p->wetting_rule != 1)
        return fail(LB_ERR_INVALID_ARG, "wetting_rule must be 0 or 1");
    return LB_OK;
}

}  // namespace

struct lb_handle {
    int n_dom = 0;
    int precision = 0, coll = 0;
    std::vector<lb_params> params;
    std::vector<DomDesc> descs;
    Layout L;
    unsigned char* base = nullptr;
    bool owns = false;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    int sm_count = 0;
    int regs_per_sm = 65536, smem_per_sm = 0, threads_per_sm = 2048;
    // Launch shape of a single domain (class 0's) and the batch schedule;
    // cls_begin / cls_count: each class's slice of the device work list.
    lb_schedule sched{};
    int cls_begin[LB_MAX_SCHED_CLASSES] = {0}, cls_count[LB_MAX_SCHED_CLASSES] = {0};
    // streams and events of the launch chains of classes 1.. in a graph
    cudaStream_t chain[LB_MAX_SCHED_CLASSES - 1] = {nullptr};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[LB_MAX_SCHED_CLASSES - 1] = {nullptr};
    int n_items = 0;
    // persistent schedules: CTAs of each class's launch
    int pgrid[LB_MAX_SCHED_CLASSES] = {0};
    // single domain: the start order of its row bands (see band_multiplier)
    int band_mul = 1;
    // compact g storage: a strip that covers its whole domain takes the
    // periodic wrap from its own stage copy and leaves the ghost columns
    // alone, so after steps they may be stale; they are refreshed before
    // another schedule (which may split a domain) or a checkpoint uses them
    bool ghosts_stale = false;
    int parity = 0;
    long long steps = 0;
    long long launches = 0;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (length, start parity)
    std::vector<double> host_pts;
    int n_geo = 0;  // domains with an obstacle map

    DomDesc* d_descs() const { return reinterpret_cast<DomDesc*>(base + L.descs); }
    WorkItem* d_items() const { return reinterpret_cast<WorkItem*>(base + L.items); }
    int* d_flags() const { return reinterpret_cast<int*>(base + L.flags); }
    int* d_dep_off() const { return reinterpret_cast<int*>(base + L.dep_off); }
    int* d_dep_idx() const { return reinterpret_cast<int*>(base + L.dep_idx); }
    double* d_partials() const { return reinterpret_cast<double*>(base + L.partials); }
    StatsOut* d_stats() const { return reinterpret_cast<StatsOut*>(base + L.stats); }
    double* d_pts() const { return reinterpret_cast<double*>(base + L.pts); }
    int* d_count() const { return reinterpret_cast<int*>(base + L.count); }
    double* d_staging() const { return reinterpret_cast<double*>(base + L.staging); }
    unsigned* d_err() const { return reinterpret_cast<unsigned*>(base + L.err); }
    // two device ints per schedule class (tile counter, finished CTAs)
    int* d_sched(int c) const { return reinterpret_cast<int*>(base + L.sched) + 2 * c; }
    int block_x() const { return sched.block_x[0]; }
    int rows() const { return sched.rows[0]; }
    size_t elem() const { return precision == LB_FP32 ? 4 : 8; }
};

namespace {

void clear_graphs(lb_handle* h)
{
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

// Class of a domain under the handle's schedule.
int class_of(const lb_handle* h, int nx)
{
    for (int c = 0; c + 1 < h->sched.n_class; ++c)
        if (nx <= h->sched.max_nx[c]) return c;
    return h->sched.n_class - 1;
}

// Dependencies of the work items of a persistent schedule (compact storage).
// Item i's step reads compact rows y0 - 2 .. y1 + 1 and f rows y0 - 1 .. y1
// of its strip and 4 columns on each side (periodic in x, and in y without
// walls), and writes rows y0 .. y1 - 1 of its strip (and, at a domain edge,
// the ghost columns the strip across the wrap reads).  It waits for every
// item of its domain whose written rows meet its read rows in its own or a
// neighbouring strip: the same items have then also finished reading what
// item i overwrites.  CSR over the whole list: dep_off[i] .. dep_off[i + 1]
// index dep_idx, whose entries are class-local item indices.
int build_deps(lb_handle* h, const std::vector<WorkItem>& items, std::vector<int>& dep_off,
               std::vector<int>& dep_idx)
{
    dep_off.assign(items.size() + 1, 0);
    dep_idx.clear();
    for (int c = 0; c < h->sched.n_class; ++c) {
        const int b0 = h->cls_begin[c], n = h->cls_count[c];
        if (n == 0) continue;
        // (domain, row block, strip) -> class-local index
        std::unordered_map<long long, int> at;
        auto key = [](int d, int b, int k) {
            return ((long long)d << 40) | ((long long)b << 20) | (long long)k;
        };
        std::vector<int> nstrip(h->n_dom, 0), width(h->n_dom, 1);
        for (int li = 0; li < n; ++li) {
            const WorkItem& w = items[b0 + li];
            if (w.x0 == 0) width[w.dom] = w.cols > 0 ? w.cols : h->sched.block_x[c];
        }
        for (int li = 0; li < n; ++li) {
            const WorkItem& w = items[b0 + li];
            const int k = w.x0 / width[w.dom];
            nstrip[w.dom] = std::max(nstrip[w.dom], k + 1);
            at[key(w.dom, w.y0 / h->sched.rows[c], k)] = li;
        }
        for (int li = 0; li < n; ++li) {
            const WorkItem& w = items[b0 + li];
            const DomDesc& D = h->descs[w.dom];
            const int rows = h->sched.rows[c];
            const int nb = (D.ny + rows - 1) / rows, K = nstrip[w.dom];
            const int b = w.y0 / rows, k = w.x0 / width[w.dom];
            const int lo = w.y0 - 2, hi = w.y0 + w.rows + 2;  // read rows [lo, hi)
            std::vector<int> mine;
            for (int db = -2; db <= 2; ++db) {
                int bb = b + db;
                if (D.walls && (bb < 0 || bb >= nb)) continue;
                bb = ((bb % nb) + nb) % nb;
                const int y0 = bb * rows, y1 = std::min(y0 + rows, D.ny);
                bool meet = false;
                for (int sh = D.walls ? 0 : -1; sh <= (D.walls ? 0 : 1) && !meet; ++sh)
                    meet = y0 + sh * D.ny < hi && y1 + sh * D.ny > lo;
                if (!meet) continue;
                for (int dk = -1; dk <= 1; ++dk) {
                    const int kk = ((k + dk) % K + K) % K;
                    auto f = at.find(key(w.dom, bb, kk));
                    if (f == at.end()) return fail(LB_ERR_INVALID_ARG, "work list is not a grid");
                    if (std::find(mine.begin(), mine.end(), f->second) == mine.end())
                        mine.push_back(f->second);
                }
            }
            if (int(mine.size()) > kMaxDeps)
                return fail(LB_ERR_INVALID_ARG, "persistent schedule: item has %d neighbours",
                            int(mine.size()));
            dep_off[b0 + li] = int(dep_idx.size());
            dep_idx.insert(dep_idx.end(), mine.begin(), mine.end());
        }
    }
    dep_off[items.size()] = int(dep_idx.size());
    return LB_OK;
}

// CTAs of each class's persistent launch.  ctas_per_sm[c] > 0 fixes them
// (per SM, at most one per item); 0 shares the GPU out so that the classes,
// launched side by side, finish together: a CTA's pace is about one row per
// pipeline iteration whatever its width, so class c gets CTAs in proportion
// to its rows (plus the pipeline's five lead-in stages per item), scaled so
// that the CTAs of all classes fill fill_pct percent of the GPU (a CTA takes
// the larger of its shares of an SM's registers, shared memory and threads).
void persist_grids(lb_handle* h, const std::vector<WorkItem>& items)
{
    double work[LB_MAX_SCHED_CLASSES] = {0}, cost[LB_MAX_SCHED_CLASSES] = {0};
    bool fixed[LB_MAX_SCHED_CLASSES] = {false};
    double room = (h->sched.fill_pct > 0 ? h->sched.fill_pct : 100) / 100.0;
    for (int c = 0; c < h->sched.n_class; ++c) {
        h->pgrid[c] = 0;
        const int n = h->cls_count[c];
        if (n == 0) continue;
        const int bx = h->sched.block_x[c];
        // a pipeline iteration of a wider CTA takes a little longer (more
        // warps meet at its barrier): measured about 1 + (NW - 3) / 23
        const double pace = (bx / 32 + 20) / 23.0;
        for (int li = 0; li < n; ++li) work[c] += (items[h->cls_begin[c] + li].rows + 5) * pace;
        int regs = 0;
        size_t smem = 0;
        double share = 1.0;
        if (lbfe::persist_footprint(h->coll, bx, &regs, &smem) == 0 && h->smem_per_sm > 0) {
            const double threads = bx + 32;
            const double warp_regs = double((regs + 7) / 8 * 8) * 32.0;  // allocated per warp
            share = std::max({warp_regs * threads / 32.0 / h->regs_per_sm,
                              double(smem + 1024) / h->smem_per_sm, threads / h->threads_per_sm});
        } else {
            share = 1.0 / std::max(1, lbfe::persist_occupancy(h->coll, bx));
        }
        cost[c] = share / h->sm_count;
        if (h->sched.ctas_per_sm[c] > 0) {
            h->pgrid[c] = std::min(h->sched.ctas_per_sm[c] * h->sm_count, n);
            fixed[c] = true;
            room -= h->pgrid[c] * cost[c];
        }
    }
    // proportional shares; a class capped at one CTA per item gives its
    // spare room back to the others
    for (int pass = 0; pass < LB_MAX_SCHED_CLASSES; ++pass) {
        double demand = 0.0;
        for (int c = 0; c < h->sched.n_class; ++c)
            if (h->cls_count[c] > 0 && !fixed[c]) demand += work[c] * cost[c];
        if (demand <= 0.0) break;
        const double alpha = std::max(room, 0.0) / demand;
        bool capped = false;
        for (int c = 0; c < h->sched.n_class; ++c) {
            if (h->cls_count[c] == 0 || fixed[c]) continue;
            if (alpha * work[c] >= h->cls_count[c]) {
                h->pgrid[c] = h->cls_count[c];
                fixed[c] = true;
                room -= h->pgrid[c] * cost[c];
                capped = true;
            }
        }
        if (capped) continue;
        for (int c = 0; c < h->sched.n_class; ++c)
            if (h->cls_count[c] > 0 && !fixed[c])
                h->pgrid[c] = std::max(1, std::min(h->cls_count[c], int(alpha * work[c] + 0.5)));
        break;
    }
}

// Start order of the row bands of a single domain's launch (band_of in the
// kernels).  About N = resident CTAs / strips bands are in flight at a time,
// and a band reads its first rows when it starts and its last ones when it
// ends, so band b should start about N grid rows after band b - 1: the rows
// both read are then read at about the same time and the second read finds
// them in L2.  Grid row g takes band g L^-1 mod B (B bands), L odd, coprime
// to B and about 3/4 of N (measured on 8192^2 with 16-row bands, N = 17.9:
// 63.4 GLUPS in order, 65.0 at L = 13, 64.5 at 17, 62.7 at 21 and beyond);
// 1 (in order) when all bands are in flight at once.  Compact storage only:
// the full-storage step measured no gain at any L (43.9 GLUPS in order,
// 42.8-44.1 strided).
int band_multiplier(const lb_handle* h)
{
    const DomDesc& D = h->descs[0];
    if (D.cls || h->n_dom != 1 || !D.compact) return 1;
    const int bx = h->block_x(), rows = h->rows();
    const int w = D.compact ? lbfe::compact_strip(bx) : bx;
    const long long strips = (D.nx + w - 1) / w, B = (D.ny + rows - 1) / rows;
    const int occ = lbfe::step_single_occupancy(h->precision, h->coll, D.compact, bx);
    const long long L = 3LL * occ * h->sm_count / (4 * std::max(strips, 1LL));
    if (L < 2 || B <= L + 1) return 1;
    for (long long l = L | 1; l < B; l += 2) {
        if (std::gcd(l, B) != 1) continue;
        // inverse of l modulo B (extended Euclid)
        long long r0 = B, r1 = l, t0 = 0, t1 = 1;
        while (r1 != 0) {
            const long long qt = r0 / r1;
            long long tmp = r0 - qt * r1;
            r0 = r1;
            r1 = tmp;
            tmp = t0 - qt * t1;
            t0 = t1;
            t1 = tmp;
        }
        return int(((t0 % B) + B) % B);
    }
    return 1;
}

// Work list for the batched kernel: every (domain, x strip, row block),
// grouped by schedule class (class c's items are one contiguous slice).
int build_items(lb_handle* h)
{
    for (int c = 0; c < LB_MAX_SCHED_CLASSES; ++c) h->cls_begin[c] = h->cls_count[c] = 0;
    if (h->n_dom == 1) {
        h->n_items = 0;
        h->band_mul = band_multiplier(h);
        return LB_OK;
    }
    std::vector<WorkItem> items;
    for (int c = 0; c < h->sched.n_class; ++c) {
        const int bx = h->sched.block_x[c], rows = h->sched.rows[c];
        std::vector<WorkItem> mine;
        for (int d = 0; d < h->n_dom; ++d) {
            const DomDesc& D = h->descs[d];
            if (D.cls || class_of(h, D.nx) != c) continue;  // obstacles: their own kernels
            if (D.compact) {
                // the compact step's strips leave room for four halo columns; a
                // domain is cut into near-equal strips (multiples of 4 columns,
                // so every bulk copy stays 16-byte aligned) instead of full
                // strips and one narrow remainder
                const int wmax = lbfe::compact_strip(bx);
                const int k = (D.nx + wmax - 1) / wmax;
                const int w = ((D.nx + k - 1) / k + 3) / 4 * 4;
                const int seal = h->sched.seal_edges[c] ? lbfe::kItemSeal : 0;
                for (int y0 = 0; y0 < D.ny; y0 += rows)
                    for (int x0 = 0; x0 < D.nx; x0 += w)
                        mine.push_back(WorkItem{d, x0, y0, std::min(rows, D.ny - y0),
                                                std::min(w, D.nx - x0), seal});
                continue;
            }
            for (int y0 = 0; y0 < D.ny; y0 += rows)
                for (int x0 = 0; x0 < D.nx; x0 += bx)
                    mine.push_back(WorkItem{d, x0, y0, std::min(rows, D.ny - y0), 0, 0});
        }
        if (h->sched.order == 1) {
            // largest first: nodes of the item (the full-storage strip is
            // bx wide, clipped to the domain)
            auto size = [&](const WorkItem& w) {
                const int cols = w.cols > 0 ? w.cols : std::min(bx, h->descs[w.dom].nx - w.x0);
                return (long long)cols * w.rows;
            };
            std::stable_sort(mine.begin(), mine.end(), [&](const WorkItem& a, const WorkItem& b) {
                return size(a) > size(b);
            });
        }
        h->cls_begin[c] = int(items.size());
        h->cls_count[c] = int(mine.size());
        items.insert(items.end(), mine.begin(), mine.end());
    }
    if ((long long)items.size() > h->L.item_cap)
        return fail(LB_ERR_INVALID_ARG, "work list exceeds its capacity");
    h->n_items = int(items.size());
    if (!items.empty())
        LB_CUDA(cudaMemcpyAsync(h->d_items(), items.data(), sizeof(WorkItem) * items.size(),
                                cudaMemcpyHostToDevice, h->stream));
    std::vector<int> dep_off, dep_idx;
    if (h->sched.persist && !items.empty()) {
        const int rc = build_deps(h, items, dep_off, dep_idx);
        if (rc != LB_OK) return rc;
        LB_CUDA(cudaMemcpyAsync(h->d_dep_off(), dep_off.data(), sizeof(int) * dep_off.size(),
                                cudaMemcpyHostToDevice, h->stream));
        LB_CUDA(cudaMemcpyAsync(h->d_dep_idx(), dep_idx.data(), sizeof(int) * dep_idx.size(),
                                cudaMemcpyHostToDevice, h->stream));
        persist_grids(h, items);
    }
    LB_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

// Grid of class c's launch: a persistent grid, or one CTA per work item.
int class_grid(const lb_handle* h, int c)
{
    const int k = h->sched.ctas_per_sm[c];
    return k > 0 ? std::min(k * h->sm_count, std::max(h->cls_count[c], 1)) : 0;
}

// The staged-kernel launch of schedule class c (batch) for one step.  With
// several classes every class launches the same kernel body, whatever its
// width: the class kernels run side by side on the SMs and then share the
// instruction caches (the 256 drops: 0.798 -> 0.805 of the copy peak with
// 64-row items, 0.81 -> 0.82 with 96; one class of 184-column strips alone
// runs 1.7 % faster on the body built for its width, which it keeps).
int launch_class(lb_handle* h, int c, int parity, cudaStream_t s)
{
    const int e = lbfe::launch_step(h->precision, h->coll, h->descs[0], h->d_descs(),
                                    h->d_items() + h->cls_begin[c], h->cls_count[c], h->n_dom,
                                    parity, h->sched.block_x[c], h->sched.rows[c], 1,
                                    class_grid(h, c), h->d_sched(c), h->sched.n_class > 1, s);
    if (e != 0)
        return fail(LB_ERR_CUDA, "step launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    return LB_OK;
}

// The persistent launch of schedule class c: `len` steps, step k reading
// buffer parity ^ (k & 1), or always `parity` with fixed_parity.
int launch_persist_class(lb_handle* h, int c, int len, int parity, bool fixed_parity,
                         cudaStream_t s)
{
    if ((long long)h->cls_count[c] * len >= (1LL << 31))
        return fail(LB_ERR_INVALID_ARG, "persistent launch: too many (step, item) tickets");
    lbfe::PersistLaunch a{};
    a.descs = h->d_descs();
    a.items = h->d_items() + h->cls_begin[c];
    a.dep_off = h->d_dep_off() + h->cls_begin[c];
    a.dep_idx = h->d_dep_idx();
    a.flags = h->d_flags() + h->cls_begin[c];
    a.sched = h->d_sched(c);
    a.err = h->d_err();
    a.n_items = h->cls_count[c];
    a.n_steps = len;
    a.parity0 = parity;
    a.flip = fixed_parity ? 0 : 1;
    a.bx = h->sched.block_x[c];
    a.grid = h->pgrid[c];
    const int e = lbfe::launch_persist(h->coll, a, s);
    if (e != 0)
        return fail(LB_ERR_CUDA, "persistent step launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    return LB_OK;
}

bool persistent(const lb_handle* h) { return h->n_dom > 1 && h->sched.persist != 0; }

// Kernel launches of one time step.
long long launches_per_step(const lb_handle* h)
{
    long long n = 0;
    if (h->n_dom == 1)
        n = h->descs[0].cls == nullptr ? 1 : 0;
    else
        for (int c = 0; c < h->sched.n_class; ++c) n += h->cls_count[c] > 0;
    return n + h->n_geo;  // one launch per domain with obstacles
}

// A domain with obstacles steps as one persistent launch per lb_step call
// (each graph of steps) when the schedule asks for it and all its tiles fit
// the GPU at once (a cooperative launch), else one launch per step.
bool geo_persistent(const lb_handle* h, const DomDesc& D)
{
    if (!h->sched.persist || !D.cls) return false;
    const int occ = lbfe::geo_persist_occupancy(h->precision, h->coll);
    return (long long)lbfe::geo_tiles(D.nx, D.ny) <= (long long)occ * h->sm_count;
}

// A single domain with obstacles may run two steps per launch; each such
// launch flips the current buffer once.
bool geo_fused(const lb_handle* h)
{
    return h->n_dom == 1 && h->descs[0].cls && h->sched.steps_per_launch == 2 &&
           !geo_persistent(h, h->descs[0]);
}

// Buffer flips of `len` steps (a two-step launch flips once).
int buffer_flips(const lb_handle* h, int len) { return geo_fused(h) ? len / 2 + (len & 1) : len; }

// `len` steps of every domain with obstacles on `s`.
int enqueue_geo_steps(lb_handle* h, int len, int parity, bool fixed_parity, cudaStream_t s)
{
    if (h->n_geo == 0) return LB_OK;
    for (int d = 0; d < h->n_dom; ++d) {
        const DomDesc& D = h->descs[d];
        if (!D.cls) continue;
        int e = 0;
        if (geo_persistent(h, D)) {
            int* flags = reinterpret_cast<int*>(h->base + h->L.geo_flags[d]);
            e = lbfe::launch_geo_persist(h->precision, h->coll, D, parity, fixed_parity ? 0 : 1, len,
                                         flags, flags + lbfe::geo_tiles(D.nx, D.ny), s);
        } else if (geo_fused(h)) {
            // pairs of steps, then a single one for an odd count
            const int pairs = len / 2;
            for (int k = 0; k < pairs && e == 0; ++k)
                e = lbfe::launch_geo_step2(h->precision, h->coll, D,
                                           fixed_parity ? parity : parity ^ (k & 1), s);
            if (e == 0 && (len & 1))
                e = lbfe::launch_geo_step(h->precision, h->coll, D,
                                          fixed_parity ? parity : parity ^ (pairs & 1), s);
        } else {
            for (int k = 0; k < len && e == 0; ++k)
                e = lbfe::launch_geo_step(h->precision, h->coll, D,
                                          fixed_parity ? parity : parity ^ (k & 1), s);
        }
        if (e != 0)
            return fail(LB_ERR_CUDA, "obstacle step launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    }
    return LB_OK;
}

int enqueue_geo(lb_handle* h, int parity, cudaStream_t s)
{
    return enqueue_geo_steps(h, 1, parity, false, s);
}

// One time step of every domain: the staged kernel for the domains without
// obstacles (one launch for a single domain; one per schedule class for a
// batch, one after the other), then one launch per domain with obstacles.
int enqueue_step(lb_handle* h, int parity, cudaStream_t s)
{
    if (h->n_dom == 1) {
        if (h->descs[0].cls == nullptr) {
            const int e = lbfe::launch_step(h->precision, h->coll, h->descs[0], h->d_descs(),
                                            nullptr, 0, 1, parity, h->block_x(), h->rows(),
                                            h->band_mul, 0, h->d_sched(0), false, s);
            if (e != 0)
                return fail(LB_ERR_CUDA, "step launch failed: %s", cudaGetErrorString(cudaError_t(e)));
        }
    } else {
        for (int c = 0; c < h->sched.n_class; ++c) {
            if (h->cls_count[c] == 0) continue;
            const int rc = persistent(h) ? launch_persist_class(h, c, 1, parity, false, s)
                                         : launch_class(h, c, parity, s);
            if (rc != LB_OK) return rc;
        }
    }
    return enqueue_geo(h, parity, s);
}

// Number of schedule classes with work.
int active_classes(const lb_handle* h)
{
    int n = 0;
    for (int c = 0; c < h->sched.n_class; ++c) n += h->cls_count[c] > 0;
    return h->n_dom == 1 ? 0 : n;
}

// Kernel launches of `len` steps (a persistent schedule runs each class's
// steps in one launch).
long long launches_for(const lb_handle* h, int len)
{
    long long geo = 0;
    for (const DomDesc& D : h->descs)
        if (D.cls) geo += geo_persistent(h, D) ? 1 : (geo_fused(h) ? len / 2 + (len & 1) : len);
    if (!persistent(h)) return len * (launches_per_step(h) - h->n_geo) + geo;
    return active_classes(h) + geo;
}

// Enqueue `len` steps on `s` (the capture stream).  With several schedule
// classes and chains on, each class runs its `len` launches as its own
// chain on its own stream, forked from `s` at the start and joined back at
// the end (the classes own disjoint domains).  fixed_parity: every step
// reads the current buffer and writes the idle one (the state does not
// advance; used to time candidates).
int enqueue_steps(lb_handle* h, int len, int parity, bool fixed_parity, cudaStream_t s)
{
    auto par = [&](int k) { return fixed_parity ? parity : parity ^ (k & 1); };
    // a class's `len` steps: one persistent launch, or a launch per step
    auto class_steps = [&](int c, cudaStream_t sc) -> int {
        if (persistent(h)) return launch_persist_class(h, c, len, parity, fixed_parity, sc);
        for (int k = 0; k < len; ++k) {
            const int rc = launch_class(h, c, par(k), sc);
            if (rc != LB_OK) return rc;
        }
        return LB_OK;
    };
    if (persistent(h) && !(h->sched.chains && active_classes(h) > 1)) {
        for (int k = 0; k < h->sched.n_class; ++k) {
            const int c = h->sched.n_class - 1 - k;
            if (h->cls_count[c] == 0) continue;
            const int rc = class_steps(c, s);
            if (rc != LB_OK) return rc;
        }
        return enqueue_geo_steps(h, len, parity, fixed_parity, s);
    }
    if (!(h->sched.chains && active_classes(h) > 1)) {
        // a single domain with obstacles: its steps, maybe in one launch
        if (h->n_dom == 1 && h->descs[0].cls) return enqueue_geo_steps(h, len, parity, fixed_parity, s);
        for (int k = 0; k < len; ++k) {
            const int rc = enqueue_step(h, par(k), s);
            if (rc != LB_OK) return rc;
        }
        return LB_OK;
    }
    LB_CUDA(cudaEventRecord(h->fork_ev, s));
    int used = 0;
    // persistent launches widest class first: its CTAs, the largest, find
    // room before the smaller ones fill the gaps
    for (int k = 0; k < h->sched.n_class; ++k) {
        const int c = persistent(h) ? h->sched.n_class - 1 - k : k;
        if (h->cls_count[c] == 0) continue;
        cudaStream_t sc = s;
        if (used > 0) {
            sc = h->chain[used - 1];
            LB_CUDA(cudaStreamWaitEvent(sc, h->fork_ev, 0));
        }
        const int rc = class_steps(c, sc);
        if (rc != LB_OK) return rc;
        if (used > 0) LB_CUDA(cudaEventRecord(h->join_ev[used - 1], sc));
        ++used;
    }
    {
        const int rc = enqueue_geo_steps(h, len, parity, fixed_parity, s);
        if (rc != LB_OK) return rc;
    }
    for (int u = 1; u < used; ++u) LB_CUDA(cudaStreamWaitEvent(s, h->join_ev[u - 1], 0));
    return LB_OK;
}

// Capture `len` steps into an executable graph.
int capture_steps(lb_handle* h, int len, int parity, bool fixed_parity, cudaGraphExec_t* out)
{
    cudaGraph_t graph = nullptr;
    LB_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_steps(h, len, parity, fixed_parity, h->cap_stream);
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
    if (rc != LB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ec != cudaSuccess) return fail(LB_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess)
        return fail(LB_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ei));
    *out = exec;
    return LB_OK;
}

int get_graph(lb_handle* h, int len, int parity, cudaGraphExec_t* out)
{
    auto key = std::make_pair(len, parity);
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        *out = it->second;
        return LB_OK;
    }
    cudaGraphExec_t exec = nullptr;
    const int rc = capture_steps(h, len, parity, false, &exec);
    if (rc != LB_OK) return rc;
    h->graphs[key] = exec;
    *out = exec;
    return LB_OK;
}

// Rewrite the periodic ghost columns of every domain's current buffer from
// the columns they copy (see lb_handle::ghosts_stale).
int refresh_ghosts(lb_handle* h)
{
    if (!h->ghosts_stale) return LB_OK;
    for (const DomDesc& D : h->descs) {
        if (D.cls) continue;
        const int e = lbfe::launch_fill_ghosts(h->precision, D, h->parity, h->stream);
        if (e != 0) return fail(LB_ERR_CUDA, "ghost refresh failed: %s", cudaGetErrorString(cudaError_t(e)));
        h->launches += 1;
    }
    LB_CUDA(cudaStreamSynchronize(h->stream));
    h->ghosts_stale = false;
    return LB_OK;
}

// Make the handle's device current for this runtime (it keeps its own
// notion of the current device, separate from other runtimes in the process).
int use_device(const lb_handle* h)
{
    if (!h) return fail(LB_ERR_INVALID_ARG, "handle is NULL");
    const cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, "cudaSetDevice failed: %s", cudaGetErrorString(e));
    return LB_OK;
}

// Synchronise the stream and report a device-side timeout recorded by a
// bounded wait (the word is cleared once reported).
int sync_and_check(lb_handle* h)
{
    unsigned err = 0;
    LB_CUDA(cudaMemcpyAsync(&err, h->d_err(), sizeof(err), cudaMemcpyDeviceToHost, h->stream));
    LB_CUDA(cudaStreamSynchronize(h->stream));
    if (err != 0) {
        cudaMemsetAsync(h->d_err(), 0, sizeof(unsigned), h->stream);
        cudaStreamSynchronize(h->stream);
        return fail(LB_ERR_TIMEOUT, "a device wait gave up (error word 0x%x)", err);
    }
    return LB_OK;
}

int check_dom(const lb_handle* h, int dom)
{
    if (!h) return fail(LB_ERR_INVALID_ARG, "handle is NULL");
    if (dom < 0 || dom >= h->n_dom) return fail(LB_ERR_INVALID_ARG, "domain %d out of range", dom);
    return use_device(h);
}

// phi0 scratch: the idle ping-pong buffer of the domain, read as doubles
double* phi0_scratch(lb_handle* h, int dom)
{
    return static_cast<double*>(h->descs[dom].f[h->parity ^ 1]);
}

int finish_init(lb_handle* h, int dom)
{
    // every domain of a handle shares one parity; the new state goes to the
    // current buffer, phi0 sat in the other one
    const DomDesc& D = h->descs[dom];
    int e;
    // phi0 is consumed once the equilibria are written: clear its scratch, so
    // that the idle buffer's padding columns, which no step reads and only
    // sealing whole-domain strips overwrite (with zeros), hold zeros whatever
    // the schedule, and checkpoints do not depend on it
    const size_t scratch = sizeof(double) * size_t(D.plane);
    if (D.cls) {
        e = lbfe::launch_geo_init_eq(h->precision, D, phi0_scratch(h, dom), h->parity, h->stream);
        if (e == 0) e = int(cudaMemsetAsync(phi0_scratch(h, dom), 0, scratch, h->stream));
        // solid nodes of the idle buffer: rest state
        if (e == 0) e = lbfe::launch_geo_solid_rest(h->precision, D, h->parity ^ 1, h->stream);
        h->launches += 2;
    } else {
        e = lbfe::launch_init_eq(h->precision, D, phi0_scratch(h, dom), h->parity, h->stream);
        if (e == 0) e = int(cudaMemsetAsync(phi0_scratch(h, dom), 0, scratch, h->stream));
        h->launches += 1;
    }
    if (e != 0) return fail(LB_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    h->steps = 0;
    return LB_OK;
}

int make_handle(const lb_params* per_dom, const int* nx, const int* ny, int n_dom, void* stream,
                void* dev_mem, size_t dev_bytes, lb_handle** out)
{
    if (!out) return fail(LB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_dom < 1 || !per_dom || !nx || !ny) return fail(LB_ERR_INVALID_ARG, "bad domain list");
    for (int d = 0; d < n_dom; ++d) {
        const int rc = validate(&per_dom[d]);
        if (rc != LB_OK) return rc;
        if (per_dom[d].precision != per_dom[0].precision ||
            per_dom[d].collision != per_dom[0].collision ||
            per_dom[d].compact_g != per_dom[0].compact_g)
            return fail(LB_ERR_INVALID_ARG,
                        "precision, collision and compact_g must match across a batch");
        if (nx[d] < 3 || ny[d] < 3) return fail(LB_ERR_INVALID_ARG, "domain %d smaller than 3x3", d);
    }
    Layout L;
    if (!build_layout(per_dom[0].precision, n_dom, nx, ny, L))
        return fail(LB_ERR_INVALID_ARG, "domain too large (9 planes must stay below 2^31 elements)");
    if (dev_mem && (dev_bytes < L.total || (reinterpret_cast<uintptr_t>(dev_mem) % kAlign) != 0))
        return fail(LB_ERR_INVALID_ARG, "dev_mem must be %zu bytes, 256-byte aligned", L.total);

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1)
        return fail(LB_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));

    int device = 0;
    if (dev_mem) {
        cudaPointerAttributes attr{};
        e = cudaPointerGetAttributes(&attr, dev_mem);
        if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice)
            return fail(LB_ERR_INVALID_ARG, "dev_mem is not device memory");
        device = attr.device;
    } else if ((e = cudaGetDevice(&device)) != cudaSuccess) {
        return fail(LB_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    }
    if ((e = cudaSetDevice(device)) != cudaSuccess)
        return fail(LB_ERR_CUDA, "cudaSetDevice(%d) failed: %s", device, cudaGetErrorString(e));

    lb_handle* h = new lb_handle();
    h->device = device;
    h->n_dom = n_dom;
    h->precision = per_dom[0].precision;
    h->coll = per_dom[0].collision;
    h->params.assign(per_dom, per_dom + n_dom);
    h->L = L;
    h->stream = static_cast<cudaStream_t>(stream);
    auto bail = [&](int rc) {
        lb_destroy(h);
        return rc;
    };
    if ((e = cudaError_t(lbfe::prepare_step_kernels())) != cudaSuccess ||
        (e = cudaError_t(lbfe::prepare_geo_step2())) != cudaSuccess)
        return bail(fail(LB_ERR_CUDA, "kernel setup failed: %s", cudaGetErrorString(e)));
    if ((e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device)) !=
            cudaSuccess ||
        (e = cudaDeviceGetAttribute(&h->regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor,
                                    h->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&h->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                    h->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&h->threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor,
                                    h->device)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(fail(LB_ERR_CUDA, "device setup failed: %s", cudaGetErrorString(e)));
    if (n_dom > 1) {
        if ((e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming)) != cudaSuccess)
            return bail(fail(LB_ERR_CUDA, "event setup failed: %s", cudaGetErrorString(e)));
        for (int c = 0; c + 1 < LB_MAX_SCHED_CLASSES; ++c)
            if ((e = cudaStreamCreateWithFlags(&h->chain[c], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h->join_ev[c], cudaEventDisableTiming)) != cudaSuccess)
                return bail(fail(LB_ERR_CUDA, "stream setup failed: %s", cudaGetErrorString(e)));
    }
    if (dev_mem) {
        h->base = static_cast<unsigned char*>(dev_mem);
        h->owns = false;
    } else {
        void* p = nullptr;
        if ((e = cudaMalloc(&p, L.total)) != cudaSuccess)
            return bail(fail(LB_ERR_CUDA, "cudaMalloc(%zu) failed: %s", L.total, cudaGetErrorString(e)));
        h->base = static_cast<unsigned char*>(p);
        h->owns = true;
    }
    for (int d = 0; d < n_dom; ++d) {
        const lb_params& p = per_dom[d];
        DomDesc D{};
        const int pitch = pitch_for(nx[d], h->precision);
        D.nx = nx[d];
        D.ny = ny[d];
        D.pitch = pitch;
        D.plane = (long long)pitch * ny[d];
        const size_t half = size_t(9) * size_t(D.plane) * h->elem();
        for (int b = 0; b < 2; ++b) {
            unsigned char* buf = h->base + L.dom_off[d] + b * L.dom_bytes[d];
            D.f[b] = buf;
            D.g[b] = buf + half;
        }
        D.walls = p.walls;
        D.step2 = p.zero_u_at_walls ? 1 : 0;
        D.step2_relax_j = p.step2_relax_momentum ? 1 : 0;
        D.compact = p.compact_g ? 1 : 0;
        D.wet_k = p.wetting_rule ? 1 : 2;
        D.a = p.a;
        D.kappa = p.kappa;
        D.gamma = p.gamma_mob;
        D.omega_phi = 1.0 / p.tau_phi;
        D.tau_c0 = p.tau_beta + 0.5 * (p.tau_alpha - p.tau_beta);
        D.tau_c1 = 0.5 * (p.tau_alpha - p.tau_beta);
        D.h_bot = p.h_bottom;
        D.h_top = p.h_top;
        D.lut_lo = D.lut_step = D.lut_inv = D.lut_kmax = 0.0;
        if (p.mrt_lut >= 2 && p.tau_alpha != p.tau_beta) {
            D.lut_lo = std::min(p.tau_alpha, p.tau_beta);
            D.lut_step = (std::max(p.tau_alpha, p.tau_beta) - D.lut_lo) / (p.mrt_lut - 1);
            D.lut_inv = 1.0 / D.lut_step;
            D.lut_kmax = p.mrt_lut - 1;
        }
        D.err = h->d_err();
        D.fa = float(D.a);
        D.fkappa = float(D.kappa);
        D.fgamma = float(D.gamma);
        D.fomega_phi = float(D.omega_phi);
        D.ftau_c0 = float(D.tau_c0);
        D.ftau_c1 = float(D.tau_c1);
        D.fh_bot = float(D.h_bot);
        D.fh_top = float(D.h_top);
        D.flut_lo = float(D.lut_lo);
        D.flut_step = float(D.lut_step);
        D.flut_inv = float(D.lut_inv);
        D.flut_kmax = float(D.lut_kmax);
        D.cls = nullptr;
        for (int k = 0; k < 8; ++k) {
            D.hcls[k] = 0.0;
            D.fhcls[k] = 0.0f;
        }
        h->descs.push_back(D);
    }
    if ((e = cudaMemsetAsync(h->base, 0, L.total, h->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h->d_descs(), h->descs.data(), sizeof(DomDesc) * n_dom,
                             cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return bail(fail(LB_ERR_CUDA, "device init failed: %s", cudaGetErrorString(e)));
    // default launch shape: 128 threads (64 with compact storage, whose
    // threads take two columns each) x 32 rows, one class, a persistent grid
    // of up to 8 CTAs per SM, items in domain order (tuned by lb_autotune)
    h->sched.n_class = 1;
    for (int c = 0; c < LB_MAX_SCHED_CLASSES; ++c) {
        h->sched.max_nx[c] = 0;
        h->sched.block_x[c] = h->descs[0].compact ? 64 : 128;
        h->sched.rows[c] = 32;
        h->sched.ctas_per_sm[c] = 8;
    }
    h->sched.order = 0;
    h->sched.chains = 1;
    const int rc = build_items(h);
    if (rc != LB_OK) return bail(rc);
    *out = h;
    return LB_OK;
}

// Least-squares circle: algebraic (Kasa) fit, then Gauss-Newton on the
// geometric residuals.  Coordinates are centred for conditioning.
bool solve3(double A[3][3], double b[3], double x[3])
{
    double M[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
        M[i][3] = b[i];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
        if (std::fabs(M[piv][c]) < 1e-300) return false;
        if (piv != c)
            for (int j = 0; j < 4; ++j) std::swap(M[c][j], M[piv][j]);
        for (int r = 0; r < 3; ++r) {
            if (r == c) continue;
            const double f = M[r][c] / M[c][c];
            for (int j = c; j < 4; ++j) M[r][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < 3; ++i) x[i] = M[i][3] / M[i][i];
    return true;
}

bool fit_circle(const std::vector<double>& pts, double& xc, double& yc, double& R)
{
    const size_t n = pts.size() / 2;
    double mx = 0, my = 0;
    for (size_t i = 0; i < n; ++i) {
        mx += pts[2 * i];
        my += pts[2 * i + 1];
    }
    mx /= double(n);
    my /= double(n);
    double A[3][3] = {{0}}, b[3] = {0}, s[3];
    for (size_t i = 0; i < n; ++i) {
        const double x = pts[2 * i] - mx, y = pts[2 * i + 1] - my;
        const double row[3] = {x, y, 1.0}, r = x * x + y * y;
        for (int j = 0; j < 3; ++j) {
            for (int k = 0; k < 3; ++k) A[j][k] += row[j] * row[k];
            b[j] += row[j] * r;
        }
    }
    if (!solve3(A, b, s)) return false;
    double cx = s[0] / 2, cy = s[1] / 2;
    double rr = std::sqrt(std::max(s[2] + cx * cx + cy * cy, 0.0));
    for (int it = 0; it < 10; ++it) {
        double JtJ[3][3] = {{0}}, Jtr[3] = {0}, d[3];
        for (size_t i = 0; i < n; ++i) {
            const double dx = pts[2 * i] - mx - cx, dy = pts[2 * i + 1] - my - cy;
            const double dist = std::sqrt(dx * dx + dy * dy);
            const double res = dist - rr;
            const double J[3] = {-dx / dist, -dy / dist, -1.0};
            for (int j = 0; j < 3; ++j) {
                for (int k = 0; k < 3; ++k) JtJ[j][k] += J[j] * J[k];
                Jtr[j] -= J[j] * res;
            }
        }
        if (!solve3(JtJ, Jtr, d)) break;
        cx += d[0];
        cy += d[1];
        rr += d[2];
    }
    xc = cx + mx;
    yc = cy + my;
    R = rr;
    return std::isfinite(xc) && std::isfinite(yc) && std::isfinite(R) && R > 0;
}

// Host check of an obstacle map (the rules of the obstacle step): classes
// in range, some fluid, node-bounce-back wall nodes only in the outer rows of
// a walled domain of at least four rows with fluid next to them, and every
// solid node next to fluid (wall rows included) has fluid mirror nodes
// s + 2d in the directions its ghost value uses.
int check_geometry(const unsigned char* cls, int nx, int ny, int walls)
{
    auto at = [&](int x, int y) {
        x = ((x % nx) + nx) % nx;
        y = ((y % ny) + ny) % ny;
        return int(cls[size_t(y) * nx + x]);
    };
    // for the mirror rule a wall node is not fluid (a mirror may not land on one)
    auto solid = [&](int x, int y) {
        if (walls && (y < 0 || y >= ny)) return true;
        return at(x, y) != 0;
    };
    long long fluid = 0;
    for (size_t k = 0; k < size_t(nx) * ny; ++k) {
        const int y = int(k / nx);
        if (cls[k] == lbfe::kNodeWall) {
            if (!walls || (y != 0 && y != ny - 1) || ny < 4)
                return fail(LB_ERR_INVALID_ARG,
                            "node %zu: wall nodes (class %d) only in the outer rows of a walled "
                            "domain of at least 4 rows", k, lbfe::kNodeWall);
            if (cls[k + (y == 0 ? nx : -nx)] != 0)
                return fail(LB_ERR_INVALID_ARG, "node %zu: a wall node needs fluid next to it", k);
            continue;
        }
        if (cls[k] > lbfe::kMaxClass)
            return fail(LB_ERR_INVALID_ARG, "class %d at node %zu exceeds %d", int(cls[k]), k,
                        lbfe::kMaxClass);
        fluid += cls[k] == 0;
    }
    if (fluid == 0) return fail(LB_ERR_INVALID_ARG, "the obstacle map has no fluid node");
    static const int AX[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    static const int DG[4][2] = {{1, 1}, {-1, -1}, {-1, 1}, {1, -1}};
    for (int y = walls ? -1 : 0; y < (walls ? ny + 1 : ny); ++y)
        for (int x = 0; x < nx; ++x) {
            if (!solid(x, y)) continue;
            // wall nodes and the solid rows beyond them take no ghost value
            if (y >= 0 && y < ny && at(x, y) == lbfe::kNodeWall) continue;
            if (y < 0 && at(x, 0) == lbfe::kNodeWall) continue;
            if (y >= ny && at(x, ny - 1) == lbfe::kNodeWall) continue;
            int n = 0;
            for (auto& d : AX)
                if (!solid(x + d[0], y + d[1])) {
                    ++n;
                    if (solid(x + 2 * d[0], y + 2 * d[1]))
                        return fail(LB_ERR_INVALID_ARG,
                                    "solid node (%d, %d): feature thinner than two nodes", x, y);
                }
            if (n > 0) continue;
            for (auto& d : DG)
                if (!solid(x + d[0], y + d[1]) && solid(x + 2 * d[0], y + 2 * d[1]))
                    return fail(LB_ERR_INVALID_ARG,
                                "solid node (%d, %d): feature thinner than two nodes", x, y);
        }
    return LB_OK;
}

// The device address of a page-locked host buffer (nullptr if the buffer is
// pageable or not known to CUDA).
double* device_alias(double* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // the query's error is not the caller's
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<double*>(a.devicePointer) : nullptr;
}

// Are all requested host outputs page-locked (and so writable by a kernel)?
bool host_mapped(double* const (&outs)[4])
{
    for (int k = 0; k < 4; ++k)
        if (outs[k] && !device_alias(outs[k])) return false;
    return true;
}

}  // namespace

extern "C" {

size_t lb_device_bytes(int precision, int n_dom, const int* nx, const int* ny)
{
    if (precision != LB_FP32 && precision != LB_FP64) return 0;
    Layout L;
    if (!build_layout(precision, n_dom, nx, ny, L)) return 0;
    return L.total;
}

int lb_create(const lb_params* p, int nx, int ny, void* stream, void* dev_mem, size_t dev_bytes,
              lb_handle** out)
{
    return make_handle(p, &nx, &ny, 1, stream, dev_mem, dev_bytes, out);
}

int lb_create_batch(const lb_params* per_dom, const int* nx, const int* ny, int n_dom, void* stream,
                    void* dev_mem, size_t dev_bytes, lb_handle** out)
{
    return make_handle(per_dom, nx, ny, n_dom, stream, dev_mem, dev_bytes, out);
}

void lb_destroy(lb_handle* h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    clear_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int c = 0; c + 1 < LB_MAX_SCHED_CLASSES; ++c) {
        if (h->chain[c]) cudaStreamDestroy(h->chain[c]);
        if (h->join_ev[c]) cudaEventDestroy(h->join_ev[c]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->owns && h->base) cudaFree(h->base);
    delete h;
}

int lb_init_drop(lb_handle* h, int dom, double R, double cx, double cy)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!std::isfinite(R) || !std::isfinite(cx) || !std::isfinite(cy))
        return fail(LB_ERR_INVALID_ARG, "drop geometry must be finite");
    const int e = lbfe::launch_init_phi_drop(h->precision, h->descs[dom], phi0_scratch(h, dom), R,
                                             cx, cy, h->stream);
    if (e != 0) return fail(LB_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    h->launches += 1;
    return finish_init(h, dom);
}

int lb_init_random(lb_handle* h, int dom, double amp, unsigned long long seed)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!std::isfinite(amp)) return fail(LB_ERR_INVALID_ARG, "amp must be finite");
    const int e = lbfe::launch_init_phi_random(h->precision, h->descs[dom], phi0_scratch(h, dom),
                                               amp, seed, h->stream);
    if (e != 0) return fail(LB_ERR_CUDA, "init launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    h->launches += 1;
    return finish_init(h, dom);
}

int lb_init_phi(lb_handle* h, int dom, const double* phi0, int on_device)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!phi0) return fail(LB_ERR_INVALID_ARG, "phi0 is NULL");
    const DomDesc& D = h->descs[dom];
    // page-locked host memory is read by a kernel through its device address
    // (one pass over the host link); other host memory goes by copy
    const double* alias = on_device ? nullptr : device_alias(const_cast<double*>(phi0));
    if (alias) {
        const int e = lbfe::launch_copy_rows(D, alias, phi0_scratch(h, dom), h->stream);
        if (e != 0) return fail(LB_ERR_CUDA, "copy launch failed: %s", cudaGetErrorString(cudaError_t(e)));
        h->launches += 1;
    } else {
        LB_CUDA(cudaMemcpy2DAsync(phi0_scratch(h, dom), sizeof(double) * D.pitch, phi0,
                                  sizeof(double) * D.nx, sizeof(double) * D.nx, D.ny,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream));
    }
    rc = finish_init(h, dom);
    if (rc != LB_OK) return rc;
    LB_CUDA(cudaStreamSynchronize(h->stream));  // phi0 may be released by the caller
    return LB_OK;
}

int lb_step(lb_handle* h, int n)
{
    if (!h) return fail(LB_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(LB_ERR_INVALID_ARG, "n must be >= 0");
    if (use_device(h) != LB_OK) return LB_ERR_CUDA;
    if (n > 0 && h->descs[0].compact) h->ghosts_stale = true;
    while (n > 0) {
        int len = n >= kGraphBig ? kGraphBig : (n >= kGraphSmall ? kGraphSmall : 1);
        if (len == 1) {
            const int rc = enqueue_step(h, h->parity, h->stream);
            if (rc != LB_OK) return rc;
        } else {
            cudaGraphExec_t g = nullptr;
            const int rc = get_graph(h, len, h->parity, &g);
            if (rc != LB_OK) return rc;
            LB_CUDA(cudaGraphLaunch(g, h->stream));
        }
        if (buffer_flips(h, len) & 1) h->parity ^= 1;
        h->steps += len;
        h->launches += launches_for(h, len);
        n -= len;
    }
    return LB_OK;
}

int lb_moments(lb_handle* h, int dom, int on_device, double* rho, double* phi, double* ux,
               double* uy, lb_stats* stats)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    const DomDesc& D = h->descs[dom];
    if (stats) {
        const int e = lbfe::launch_moments(h->precision, D, h->parity, 0, D.ny, nullptr, nullptr,
                                           nullptr, nullptr, D.nx, h->d_partials(),
                                           lbfe::max_partials_needed(0, 0), h->d_stats(), h->stream);
        if (e != 0) return fail(LB_ERR_CUDA, "moments launch failed: %s", cudaGetErrorString(cudaError_t(e)));
        h->launches += 2;
    }
    double* outs[4] = {rho, phi, ux, uy};
    const bool any = rho || phi || ux || uy;
    if (any && on_device) {
        const int e = lbfe::launch_moments(h->precision, D, h->parity, 0, D.ny, rho, phi, ux, uy,
                                           D.nx, nullptr, 0, nullptr, h->stream);
        if (e != 0) return fail(LB_ERR_CUDA, "moments launch failed: %s", cudaGetErrorString(cudaError_t(e)));
        h->launches += 1;
    } else if (any && host_mapped(outs)) {
        // page-locked host buffers are mapped into the device's address
        // space: the kernel writes them directly, in one pass
        double* dev[4];
        for (int k = 0; k < 4; ++k) dev[k] = outs[k] ? device_alias(outs[k]) : nullptr;
        const int e = lbfe::launch_moments(h->precision, D, h->parity, 0, D.ny, dev[0], dev[1],
                                           dev[2], dev[3], D.nx, nullptr, 0, nullptr, h->stream);
        if (e != 0) return fail(LB_ERR_CUDA, "moments launch failed: %s", cudaGetErrorString(cudaError_t(e)));
        h->launches += 1;
    } else if (any) {
        const int chunk_rows = int(std::max<long long>(1, h->L.staging_nodes / D.nx));
        double* st = h->d_staging();
        const long long sn = h->L.staging_nodes;
        for (int r0 = 0; r0 < D.ny; r0 += chunk_rows) {
            const int nr = std::min(chunk_rows, D.ny - r0);
            double* dev[4];
            for (int k = 0; k < 4; ++k) dev[k] = outs[k] ? st + k * sn : nullptr;
            const int e = lbfe::launch_moments(h->precision, D, h->parity, r0, nr, dev[0], dev[1],
                                               dev[2], dev[3], D.nx, nullptr, 0, nullptr, h->stream);
            if (e != 0) return fail(LB_ERR_CUDA, "moments launch failed: %s", cudaGetErrorString(cudaError_t(e)));
            h->launches += 1;
            for (int k = 0; k < 4; ++k)
                if (outs[k])
                    LB_CUDA(cudaMemcpyAsync(outs[k] + (long long)r0 * D.nx, dev[k],
                                            sizeof(double) * nr * D.nx, cudaMemcpyDeviceToHost,
                                            h->stream));
        }
    }
    StatsOut so{};
    if (stats)
        LB_CUDA(cudaMemcpyAsync(&so, h->d_stats(), sizeof(StatsOut), cudaMemcpyDeviceToHost, h->stream));
    rc = sync_and_check(h);
    if (rc != LB_OK) return rc;
    if (stats) {
        stats->mass = so.mass;
        stats->order = so.order;
        stats->mom_x = so.mom_x;
        stats->mom_y = so.mom_y;
        stats->max_u = so.max_u;
        stats->nonfinite = (long long)so.nonfinite;
        stats->step = h->steps;
        if (so.nonfinite > 0)
            return fail(LB_ERR_NONFINITE, "%lld nodes with non-finite moments", stats->nonfinite);
    }
    return LB_OK;
}

int lb_contact_angle(lb_handle* h, int dom, double exclude, double* theta_deg, double* R,
                     double* xc, double* yc)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!std::isfinite(exclude)) return fail(LB_ERR_INVALID_ARG, "exclude must be finite");
    const DomDesc& D = h->descs[dom];
    const int cap = 16 * (D.nx + D.ny);
    const int e = lbfe::launch_crossings(h->precision, D, h->parity, h->d_pts(), h->d_count(), cap,
                                         h->stream);
    if (e != 0) return fail(LB_ERR_CUDA, "crossings launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    h->launches += 1;
    int count = 0;
    LB_CUDA(cudaMemcpyAsync(&count, h->d_count(), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LB_CUDA(cudaStreamSynchronize(h->stream));
    if (count > cap) return fail(LB_ERR_CAPACITY, "%d interface points exceed capacity %d", count, cap);
    std::vector<double> raw(2 * size_t(count));
    if (count > 0) {
        LB_CUDA(cudaMemcpyAsync(raw.data(), h->d_pts(), sizeof(double) * 2 * count,
                                cudaMemcpyDeviceToHost, h->stream));
        LB_CUDA(cudaStreamSynchronize(h->stream));
    }
    std::vector<std::pair<double, double>> pts;
    const double wall = -0.5;
    for (int i = 0; i < count; ++i)
        if (raw[2 * i + 1] >= wall + exclude) pts.emplace_back(raw[2 * i], raw[2 * i + 1]);
    std::sort(pts.begin(), pts.end());
    if (pts.size() < 3) return fail(LB_ERR_NO_INTERFACE, "only %zu interface points", pts.size());
    std::vector<double> flat;
    flat.reserve(2 * pts.size());
    for (auto& q : pts) {
        flat.push_back(q.first);
        flat.push_back(q.second);
    }
    double cx, cy, rr;
    if (!fit_circle(flat, cx, cy, rr)) return fail(LB_ERR_NO_INTERFACE, "circle fit failed");
    const double s = std::max(-1.0, std::min(1.0, (cy - wall) / rr));
    if (theta_deg) *theta_deg = 90.0 + std::asin(s) * 180.0 / M_PI;
    if (R) *R = rr;
    if (xc) *xc = cx;
    if (yc) *yc = cy;
    return LB_OK;
}

int lb_set_geometry(lb_handle* h, int dom, const unsigned char* cls, const double* h_class,
                    int n_class)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    DomDesc& D = h->descs[dom];
    if (cls && D.compact)
        return fail(LB_ERR_INVALID_ARG, "obstacles need the full g storage (compact_g = 0)");
    if (cls) {
        if (!h_class || n_class < 1 || n_class > lbfe::kMaxClass + 1)
            return fail(LB_ERR_INVALID_ARG, "h_class must hold 1..%d entries", lbfe::kMaxClass + 1);
        for (int k = 0; k < n_class; ++k)
            if (!std::isfinite(h_class[k]))
                return fail(LB_ERR_INVALID_ARG, "wetting gradient of class %d is not finite", k);
        for (size_t q = 0; q < size_t(D.nx) * D.ny; ++q)
            if (cls[q] >= n_class && cls[q] != lbfe::kNodeWall)
                return fail(LB_ERR_INVALID_ARG, "node %zu has class %d but only %d classes given",
                            q, int(cls[q]), n_class);
        rc = check_geometry(cls, D.nx, D.ny, D.walls);
        if (rc != LB_OK) return rc;
    }
    LB_CUDA(cudaStreamSynchronize(h->stream));
    clear_graphs(h);
    unsigned char* dev = h->base + h->L.geo_off[dom];
    const bool had = D.cls != nullptr;
    if (cls) {
        LB_CUDA(cudaMemcpyAsync(dev, cls, size_t(D.nx) * D.ny, cudaMemcpyHostToDevice, h->stream));
        D.cls = dev;
        for (int k = 0; k < 8; ++k) {
            D.hcls[k] = k < n_class ? h_class[k] : 0.0;
            D.fhcls[k] = float(D.hcls[k]);
        }
    } else {
        D.cls = nullptr;
    }
    h->n_geo += (D.cls != nullptr) - int(had);
    LB_CUDA(cudaMemcpyAsync(h->d_descs() + dom, &D, sizeof(DomDesc), cudaMemcpyHostToDevice,
                            h->stream));
    LB_CUDA(cudaStreamSynchronize(h->stream));
    return build_items(h);
}

int lb_set_wetting(lb_handle* h, int dom, double h_bottom, double h_top)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!std::isfinite(h_bottom) || !std::isfinite(h_top))
        return fail(LB_ERR_INVALID_ARG, "wetting gradients must be finite");
    DomDesc& D = h->descs[dom];
    // kernels take the descriptor by value (captured in the step graphs)
    LB_CUDA(cudaStreamSynchronize(h->stream));
    clear_graphs(h);
    h->params[dom].h_bottom = h_bottom;
    h->params[dom].h_top = h_top;
    D.h_bot = h_bottom;
    D.h_top = h_top;
    D.fh_bot = float(h_bottom);
    D.fh_top = float(h_top);
    LB_CUDA(cudaMemcpyAsync(h->d_descs() + dom, &D, sizeof(DomDesc), cudaMemcpyHostToDevice,
                            h->stream));
    LB_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_get_geometry(lb_handle* h, int dom, unsigned char* cls)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!cls) return fail(LB_ERR_INVALID_ARG, "cls is NULL");
    const DomDesc& D = h->descs[dom];
    if (!D.cls) {
        memset(cls, 0, size_t(D.nx) * D.ny);
        return LB_OK;
    }
    LB_CUDA(cudaMemcpyAsync(cls, D.cls, size_t(D.nx) * D.ny, cudaMemcpyDeviceToHost, h->stream));
    LB_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_init_channel(lb_handle* h, int dom, int res_len, int ch_w, double h_channel,
                    double h_block)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    const DomDesc& D0 = h->descs[dom];
    const int nx = D0.nx, ny = D0.ny;
    if (!D0.walls) return fail(LB_ERR_INVALID_ARG, "the capillary set-up needs walls");
    if (res_len < 4 || nx - res_len < 1)
        return fail(LB_ERR_INVALID_ARG, "res_len must be in [4, nx - 1]");
    const int y0 = (ny - ch_w) / 2;
    if (ch_w < 2 || y0 < 1 || y0 + ch_w + 1 > ny)
        return fail(LB_ERR_INVALID_ARG, "channel width must leave a solid row on each side");
    if (!std::isfinite(h_channel) || !std::isfinite(h_block))
        return fail(LB_ERR_INVALID_ARG, "wetting gradients must be finite");
    std::vector<unsigned char> cls(size_t(nx) * ny, 0);
    for (int y = 0; y < ny; ++y)
        for (int x = res_len; x < nx; ++x) {
            unsigned char c = 2;
            if (y >= y0 && y < y0 + ch_w) c = 0;
            if (y == y0 - 1 || y == y0 + ch_w) c = 1;
            cls[size_t(y) * nx + x] = c;
        }
    const double hc[3] = {0.0, h_channel, h_block};
    rc = lb_set_geometry(h, dom, cls.data(), hc, 3);
    if (rc != LB_OK) return rc;
    // phase alpha in the reservoir columns [res_len/2, res_len), beta elsewhere;
    // flat tanh profiles centred half a node before each interface column
    const DomDesc& D = h->descs[dom];
    const double l = std::sqrt(2.0 * D.kappa / D.a);
    const double xa = res_len / 2 - 0.5, xb = res_len - 0.5;
    std::vector<double> phi0(size_t(nx) * ny);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t k = size_t(y) * nx + x;
            phi0[k] = cls[k] ? 0.0 : std::tanh(std::min(x - xa, xb - x) / l);
        }
    return lb_init_phi(h, dom, phi0.data(), 0);
}

int lb_meniscus(lb_handle* h, int dom, int x_lo, int x_hi, int y_lo, int y_hi, double exclude,
                double* x_front, double* theta_deg, double* R)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    const DomDesc& D = h->descs[dom];
    if (x_lo < 0 || x_hi > D.nx || x_lo + 2 > x_hi || y_lo < 0 || y_hi > D.ny || y_lo + 2 > y_hi ||
        !std::isfinite(exclude))
        return fail(LB_ERR_INVALID_ARG, "bad meniscus box");
    const int cap = 16 * (D.nx + D.ny);
    const int e = lbfe::launch_crossings(h->precision, D, h->parity, h->d_pts(), h->d_count(), cap,
                                         h->stream);
    if (e != 0) return fail(LB_ERR_CUDA, "crossings launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    h->launches += 1;
    int count = 0;
    LB_CUDA(cudaMemcpyAsync(&count, h->d_count(), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LB_CUDA(cudaStreamSynchronize(h->stream));
    if (count > cap) return fail(LB_ERR_CAPACITY, "%d interface points exceed capacity %d", count, cap);
    std::vector<double> raw(2 * size_t(count));
    if (count > 0) {
        LB_CUDA(cudaMemcpyAsync(raw.data(), h->d_pts(), sizeof(double) * 2 * count,
                                cudaMemcpyDeviceToHost, h->stream));
        LB_CUDA(cudaStreamSynchronize(h->stream));
    }
    // points on links with both ends in the box, away from the walls
    const double wb = y_lo - 0.5, wt = y_hi - 0.5;
    std::vector<std::pair<double, double>> pts;
    for (int i = 0; i < count; ++i) {
        const double px = raw[2 * i], py = raw[2 * i + 1];
        if (px < x_lo || px > x_hi - 1 || py < y_lo || py > y_hi - 1) continue;
        if (py < wb + exclude || py > wt - exclude) continue;
        pts.emplace_back(px, py);
    }
    std::sort(pts.begin(), pts.end());
    if (pts.size() < 3) return fail(LB_ERR_NO_INTERFACE, "only %zu meniscus points", pts.size());
    std::vector<double> flat;
    double mx = 0.0;
    for (auto& q : pts) {
        flat.push_back(q.first);
        flat.push_back(q.second);
        mx += q.first;
    }
    mx /= double(pts.size());
    double cx, cy, rr;
    if (!fit_circle(flat, cx, cy, rr)) return fail(LB_ERR_NO_INTERFACE, "circle fit failed");
    // centre ahead of the points (beta side): alpha wets the walls
    const double sg = cx > mx ? 1.0 : -1.0;
    auto clampc = [](double v) { return std::max(-1.0, std::min(1.0, v)); };
    const double tb = std::acos(clampc(sg * (cy - wb) / rr)), tt = std::acos(clampc(sg * (wt - cy) / rr));
    const double ym = 0.5 * (wb + wt);
    if (x_front) *x_front = cx - sg * std::sqrt(std::max(rr * rr - (ym - cy) * (ym - cy), 0.0));
    if (theta_deg) *theta_deg = 0.5 * (tb + tt) * 180.0 / M_PI;
    if (R) *R = rr;
    return LB_OK;
}

double lb_wetting_h(double theta_deg, double a, double kappa)
{
    if (!(theta_deg >= 0.0 && theta_deg <= 180.0) || !(a > 0.0) || !(kappa > 0.0)) return NAN;
    const double th = theta_deg * M_PI / 180.0;
    const double s = std::sin(th);
    const double alpha = std::acos(std::min(1.0, s * s));
    const double c = std::cos(alpha / 3.0);
    const double sgn = theta_deg > 90.0 ? 1.0 : (theta_deg < 90.0 ? -1.0 : 0.0);
    return 2.0 * sgn * std::sqrt(std::max(c * (1.0 - c), 0.0)) / std::sqrt(2.0 * kappa / a);
}

int lb_get_populations_rows(lb_handle* h, int dom, int y0, int nrows, double* f, double* g)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!f && !g) return fail(LB_ERR_INVALID_ARG, "f and g are NULL");
    const DomDesc& D = h->descs[dom];
    if (y0 < 0 || nrows < 1 || y0 + nrows > D.ny) return fail(LB_ERR_INVALID_ARG, "bad row range");
    const size_t nn = size_t(D.nx) * nrows, es = h->elem();
    std::vector<unsigned char> tmp(nn * es);
    if (D.compact && g) {
        // g' from the compact state: g'_i = g^eq_i(phi, Gamma mu, u_eq) for
        // i > 0 (Appendix A), g'_0 = phi - sum_{i>0} g'_i
        std::vector<float> c(4 * nn);
        for (int k = 0; k < 4; ++k) {
            const unsigned char* plane = static_cast<const unsigned char*>(D.g[h->parity]) +
                                         (size_t(k) * D.plane + size_t(y0) * D.pitch + lbfe::kXOff) * es;
            LB_CUDA(cudaMemcpy2DAsync(c.data() + k * nn, es * D.nx, plane, es * D.pitch,
                                      es * D.nx, nrows, cudaMemcpyDeviceToHost, h->stream));
        }
        LB_CUDA(cudaStreamSynchronize(h->stream));
        for (size_t q = 0; q < nn; ++q) {
            const double phi = lbfe::G0<float>::decode(c[q]);
            const double G = c[nn + q], ux = c[2 * nn + q], uy = c[3 * nn + q];
            const double pux = phi * ux, puy = phi * uy;
            const double pxx = pux * ux, pyy = puy * uy, pxy = pux * uy, puu = pxx + pyy;
            const double Cx = 4 * G + 6 * pxx - 2 * puu, Cy = 4 * G + 6 * pyy - 2 * puu;
            const double Cd = G + puu + 3 * pxy, Ca = G + puu - 3 * pxy;
            const double ge[9] = {0.0,
                                  (Cx + 4 * pux) / 12, (Cx - 4 * pux) / 12,
                                  (Cy + 4 * puy) / 12, (Cy - 4 * puy) / 12,
                                  (Cd + (pux + puy)) / 12, (Cd - (pux + puy)) / 12,
                                  (Ca + (puy - pux)) / 12, (Ca - (puy - pux)) / 12};
            double tail = 0.0;
            for (int i = 1; i < 9; ++i) {
                g[i * nn + q] = ge[i];
                tail += ge[i];
            }
            g[q] = phi - tail;
        }
    }
    for (int which = 0; which < 2; ++which) {
        double* out = which == 0 ? f : g;
        if (!out || (which == 1 && D.compact)) continue;
        const unsigned char* src =
            static_cast<const unsigned char*>(which == 0 ? D.f[h->parity] : D.g[h->parity]);
        for (int i = 0; i < 9; ++i) {
            const unsigned char* plane =
                src + (size_t(i) * D.plane + size_t(y0) * D.pitch + lbfe::kXOff) * es;
            LB_CUDA(cudaMemcpy2DAsync(tmp.data(), es * D.nx, plane, es * D.pitch, es * D.nx, nrows,
                                      cudaMemcpyDeviceToHost, h->stream));
            LB_CUDA(cudaStreamSynchronize(h->stream));
            const double rest = which == 0 ? kRest[i] : 0.0;
            double* o = out + i * nn;
            if (es == 4 && which == 1 && i == 0) {
                const float* t = reinterpret_cast<const float*>(tmp.data());
                for (size_t k = 0; k < nn; ++k) o[k] = lbfe::G0<float>::decode(t[k]);
            } else if (es == 4) {
                const float* t = reinterpret_cast<const float*>(tmp.data());
                for (size_t k = 0; k < nn; ++k) o[k] = rest + double(t[k]);
            } else {
                const double* t = reinterpret_cast<const double*>(tmp.data());
                for (size_t k = 0; k < nn; ++k) o[k] = rest + t[k];
            }
        }
    }
    return LB_OK;
}

int lb_get_populations(lb_handle* h, int dom, double* f, double* g)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    return lb_get_populations_rows(h, dom, 0, h->descs[dom].ny, f, g);
}

int lb_set_populations(lb_handle* h, int dom, const double* f, const double* g)
{
    int rc = check_dom(h, dom);
    if (rc != LB_OK) return rc;
    if (!f || !g) return fail(LB_ERR_INVALID_ARG, "f and g are required");
    const DomDesc& D = h->descs[dom];
    if (D.compact)
        return fail(LB_ERR_INVALID_ARG,
                    "a compact-g handle holds only equilibrium g; set its state with lb_init_* "
                    "or lb_load_state");
    const size_t nn = size_t(D.nx) * D.ny, es = h->elem();
    std::vector<unsigned char> tmp(9 * nn * es);
    for (int which = 0; which < 2; ++which) {
        const double* in = which == 0 ? f : g;
        for (int i = 0; i < 9; ++i) {
            const double rest = which == 0 ? kRest[i] : 0.0;
            for (size_t k = 0; k < nn; ++k) {
                const size_t q = i * nn + k;
                const double v = in[q] - rest;
                if (es == 4 && which == 1 && i == 0)
                    reinterpret_cast<float*>(tmp.data())[q] = lbfe::G0<float>::encode(v);
                else if (es == 4)
                    reinterpret_cast<float*>(tmp.data())[q] = float(v);
                else
                    reinterpret_cast<double*>(tmp.data())[q] = v;
            }
        }
        unsigned char* dst = static_cast<unsigned char*>(which == 0 ? D.f[h->parity] : D.g[h->parity]);
        LB_CUDA(cudaMemcpy2DAsync(dst + lbfe::kXOff * es, es * D.pitch, tmp.data(), es * D.nx,
                                  es * D.nx, 9 * D.ny, cudaMemcpyHostToDevice, h->stream));
        LB_CUDA(cudaStreamSynchronize(h->stream));
    }
    const int e = lbfe::launch_fill_ghosts(h->precision, D, h->parity, h->stream);
    if (e != 0) return fail(LB_ERR_CUDA, "ghost fill failed: %s", cudaGetErrorString(cudaError_t(e)));
    h->launches += 1;
    LB_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

size_t lb_state_bytes(const lb_handle* h)
{
    if (!h) return 0;
    size_t total = 4 * sizeof(long long);
    for (int d = 0; d < h->n_dom; ++d) total += size_t(18) * size_t(h->descs[d].plane) * h->elem();
    return total;
}

int lb_save_state(lb_handle* h, void* host_buf, size_t bytes)
{
    if (!h || !host_buf) return fail(LB_ERR_INVALID_ARG, "NULL argument");
    if (use_device(h) != LB_OK) return LB_ERR_CUDA;
    if (bytes < lb_state_bytes(h)) return fail(LB_ERR_INVALID_ARG, "buffer too small");
    const int rg = refresh_ghosts(h);  // the saved state holds current ghost columns
    if (rg != LB_OK) return rg;
    long long* hdr = static_cast<long long*>(host_buf);
    hdr[0] = 0x4c4246454348LL;  // magic
    hdr[1] = h->n_dom;
    hdr[2] = h->precision;
    hdr[3] = h->steps;
    unsigned char* p = static_cast<unsigned char*>(host_buf) + 4 * sizeof(long long);
    for (int d = 0; d < h->n_dom; ++d) {
        const size_t half = size_t(9) * size_t(h->descs[d].plane) * h->elem();
        LB_CUDA(cudaMemcpyAsync(p, h->descs[d].f[h->parity], half, cudaMemcpyDeviceToHost, h->stream));
        LB_CUDA(cudaMemcpyAsync(p + half, h->descs[d].g[h->parity], half, cudaMemcpyDeviceToHost,
                                h->stream));
        p += 2 * half;
    }
    LB_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_load_state(lb_handle* h, const void* host_buf, size_t bytes)
{
    if (!h || !host_buf) return fail(LB_ERR_INVALID_ARG, "NULL argument");
    if (use_device(h) != LB_OK) return LB_ERR_CUDA;
    if (bytes < lb_state_bytes(h)) return fail(LB_ERR_INVALID_ARG, "buffer too small");
    const long long* hdr = static_cast<const long long*>(host_buf);
    if (hdr[0] != 0x4c4246454348LL || hdr[1] != h->n_dom || hdr[2] != h->precision)
        return fail(LB_ERR_INVALID_ARG, "checkpoint does not match this handle");
    const unsigned char* p = static_cast<const unsigned char*>(host_buf) + 4 * sizeof(long long);
    for (int d = 0; d < h->n_dom; ++d) {
        const size_t half = size_t(9) * size_t(h->descs[d].plane) * h->elem();
        LB_CUDA(cudaMemcpyAsync(h->descs[d].f[h->parity], p, half, cudaMemcpyHostToDevice, h->stream));
        LB_CUDA(cudaMemcpyAsync(h->descs[d].g[h->parity], p + half, half, cudaMemcpyHostToDevice,
                                h->stream));
        p += 2 * half;
    }
    LB_CUDA(cudaStreamSynchronize(h->stream));
    h->steps = hdr[3];
    h->ghosts_stale = false;
    return LB_OK;
}

int lb_set_tile(lb_handle* h, int block_x, int rows)
{
    if (use_device(h) != LB_OK) return h ? LB_ERR_CUDA : LB_ERR_INVALID_ARG;
    lb_schedule sc = h->sched;
    sc.n_class = 1;
    sc.block_x[0] = block_x;
    sc.rows[0] = rows;
    return lb_set_schedule(h, &sc);
}

int lb_get_tile(const lb_handle* h, int* block_x, int* rows)
{
    if (!h) return fail(LB_ERR_INVALID_ARG, "handle is NULL");
    if (block_x) *block_x = h->block_x();
    if (rows) *rows = h->rows();
    return LB_OK;
}

int lb_set_schedule(lb_handle* h, const lb_schedule* sc)
{
    if (use_device(h) != LB_OK) return h ? LB_ERR_CUDA : LB_ERR_INVALID_ARG;
    if (!sc) return fail(LB_ERR_INVALID_ARG, "schedule is NULL");
    if (sc->n_class < 1 || sc->n_class > LB_MAX_SCHED_CLASSES)
        return fail(LB_ERR_INVALID_ARG, "n_class must be in [1, %d]", LB_MAX_SCHED_CLASSES);
    for (int c = 0; c < sc->n_class; ++c) {
        const int bx = sc->block_x[c];
        // compact storage takes strips of up to nine compute warps (556 columns)
        const int max_bx = h->descs[0].compact ? kMaxBlockXCompact : kMaxBlockX;
        if (bx < kMinBlockX || bx > max_bx || bx % 32 != 0 || sc->rows[c] < 1 ||
            (!h->descs[0].compact && lbfe::step_smem_bytes(h->precision, bx) == 0))
            return fail(LB_ERR_INVALID_ARG,
                        "block_x must be a multiple of 32 in [32, %d], rows >= 1 (class %d)", max_bx,
                        c);
        if (sc->ctas_per_sm[c] < 0 || sc->ctas_per_sm[c] > 32)
            return fail(LB_ERR_INVALID_ARG, "ctas_per_sm must be in [0, 32] (class %d)", c);
        if (sc->seal_edges[c] != 0 && sc->seal_edges[c] != 1)
            return fail(LB_ERR_INVALID_ARG, "seal_edges must be 0 or 1 (class %d)", c);
        if (c + 1 < sc->n_class &&
            (sc->max_nx[c] < 1 || (c > 0 && sc->max_nx[c] <= sc->max_nx[c - 1])))
            return fail(LB_ERR_INVALID_ARG, "max_nx must be positive and increasing");
    }
    if ((sc->order != 0 && sc->order != 1) || (sc->chains != 0 && sc->chains != 1) ||
        (sc->persist != 0 && sc->persist != 1))
        return fail(LB_ERR_INVALID_ARG, "order, chains and persist must be 0 or 1");
    if (sc->fill_pct < 0 || sc->fill_pct > 400)
        return fail(LB_ERR_INVALID_ARG, "fill_pct must be in [0, 400]");
    if (sc->steps_per_launch < 0 || sc->steps_per_launch > 2)
        return fail(LB_ERR_INVALID_ARG, "steps_per_launch must be 0, 1 or 2");

    if (sc->persist && h->n_dom > 1 && !(h->precision == LB_FP32 && h->descs[0].compact))
        return fail(LB_ERR_INVALID_ARG, "persistent schedules need compact FP32 storage");
    const int rg = refresh_ghosts(h);  // the new schedule may split a domain into strips
    if (rg != LB_OK) return rg;
    LB_CUDA(cudaStreamSynchronize(h->stream));
    clear_graphs(h);
    lb_schedule v = *sc;
    for (int c = v.n_class; c < LB_MAX_SCHED_CLASSES; ++c) {  // unused classes: class 0's values
        v.max_nx[c] = 0;
        v.block_x[c] = v.block_x[0];
        v.rows[c] = v.rows[0];
        v.ctas_per_sm[c] = v.ctas_per_sm[0];
        v.seal_edges[c] = v.seal_edges[0];
    }
    v.max_nx[v.n_class - 1] = 0;
    h->sched = v;
    return build_items(h);
}

int lb_get_schedule(const lb_handle* h, lb_schedule* sc)
{
    if (!h || !sc) return fail(LB_ERR_INVALID_ARG, "NULL argument");
    *sc = h->sched;
    return LB_OK;
}

namespace {

// Device time per step of `len` fixed-parity steps (the state does not
// advance), replayed `reps` times from a captured graph after one warm-up
// replay.  Returns a negative value on failure (the error is recorded).
double time_graph_steps(lb_handle* h, int len, int reps, cudaEvent_t e0, cudaEvent_t e1)
{
    cudaGraphExec_t g = nullptr;
    if (capture_steps(h, len, h->parity, true, &g) != LB_OK) return -1.0;
    double ms_step = -1.0;
    if (cudaGraphLaunch(g, h->stream) == cudaSuccess && cudaEventRecord(e0, h->stream) == cudaSuccess) {
        bool ok = true;
        for (int k = 0; k < reps && ok; ++k) ok = cudaGraphLaunch(g, h->stream) == cudaSuccess;
        float ms = 0.f;
        if (ok && cudaEventRecord(e1, h->stream) == cudaSuccess &&
            cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
            ms_step = double(ms) / (double(reps) * len);
        else
            fail(LB_ERR_CUDA, "autotune timing failed");
    } else {
        fail(LB_ERR_CUDA, "autotune launch failed");
    }
    cudaGraphExecDestroy(g);
    h->launches += (long long)(reps + 1) * launches_for(h, len);
    return ms_step;
}

// Candidate schedules of a batch.
//  - One class: every strip width, rows per item, a persistent or one-CTA-
//    per-item grid, and the item order.
//  - Ladders of size classes: a class per strip width, each taking the
//    domains that fit one of its strips (so that with compact storage a
//    domain is one strip, which wraps in shared memory and writes no ghost
//    columns), as independent chains, largest item first, with taller
//    items (fewer halo rows per node).
std::vector<lb_schedule> batch_candidates(const lb_handle* h)
{
    const bool compact = h->descs[0].compact != 0;
    std::vector<int> widths = compact ? std::vector<int>{64, 96, 128} : std::vector<int>{64, 128, 256};
    if (h->precision == LB_FP64) widths = {64, 128};
    std::vector<lb_schedule> out;
    auto occ = [&](int bx) {
        return std::max(1, lbfe::step_batch_occupancy(h->precision, h->coll, compact, bx));
    };
    for (int bx : widths)
        for (int r : {16, 32, 64})
            for (int persistent = 0; persistent < 2; ++persistent)
                for (int order = 0; order < 2; ++order) {
                    lb_schedule s{};
                    s.n_class = 1;
                    s.chains = 1;
                    s.block_x[0] = bx;
                    s.rows[0] = r;
                    s.ctas_per_sm[0] = persistent ? occ(bx) : 0;
                    s.order = order;
                    out.push_back(s);
                }
    std::vector<std::vector<int>> ladders;
    if (compact)
        ladders = {{96, 160, 224, 288},
                   {96, 160, 192, 224, 288},
                   {96, 128, 160, 192, 224, 256, 288},
                   {64, 96, 128, 160, 192, 224, 256, 288}};
    else if (h->precision == LB_FP32)
        ladders = {{64, 128, 256}, {64, 128, 192, 256}};
    else
        ladders = {{64, 128}};
    // seal: the classes of at most `seal` compute warps seal their rows (0
    // none): the narrow strips, whose rows are short, gain the most from it
    auto ladder = [&](const std::vector<int>& lad, int r, int persist, int seal) {
        lb_schedule s{};
        s.n_class = int(lad.size());
        s.chains = 1;
        s.order = 1;
        s.persist = persist;
        s.fill_pct = persist ? 85 : 0;
        for (int c = 0; c < s.n_class; ++c) {
            s.block_x[c] = lad[c];
            s.rows[c] = r;
            s.ctas_per_sm[c] = 0;
            s.max_nx[c] = compact ? lbfe::compact_strip(lad[c]) : lad[c];
            s.seal_edges[c] = lad[c] / 32 <= seal;
        }
        out.push_back(s);
    };
    for (const auto& lad : ladders)
        for (int r : {48, 64, 96, 128}) ladder(lad, r, 0, 0);
    if (compact && h->precision == LB_FP32)
        for (const auto& lad : ladders) {
            // the same ladders with sealed rows (strips up to 184 or 244
            // columns, or all), and as persistent launches (each class's
            // steps in one launch, the GPU shared out between the classes)
            for (int r : {32, 64, 96})
                for (int seal : {3, 4, 9}) ladder(lad, r, 0, seal);
            for (int r : {32, 64}) ladder(lad, r, 1, 0);
        }
    return out;
}

}  // namespace

int lb_autotune(lb_handle* h, int reps, int* block_x, int* rows, double* best_ms)
{
    if (use_device(h) != LB_OK) return h ? LB_ERR_CUDA : LB_ERR_INVALID_ARG;
    if (reps < 1) reps = 1;
    int max_ny = 0;
    for (auto& D : h->descs) max_ny = std::max(max_ny, D.ny);
    // with obstacles only, no domain uses the staged kernel; a single domain
    // with obstacles chooses between per-step and persistent launches
    const bool plain = h->n_dom == 1 ? h->descs[0].cls == nullptr : h->n_items > 0;
    std::vector<lb_schedule> cands;
    if (!plain) {
        cands.push_back(h->sched);
        if (h->n_dom == 1) {
            // one domain with obstacles: a launch per step, two steps per
            // launch, or its steps in one persistent launch
            cands.clear();
            for (int mode = 0; mode < 3; ++mode) {
                lb_schedule p = h->sched;
                p.persist = mode == 2;
                p.steps_per_launch = mode == 1 ? 2 : 1;
                cands.push_back(p);
            }
        }
    } else if (h->n_dom > 1) {
        cands = batch_candidates(h);
    } else {
        // compact storage: two columns per thread, so half the threads per
        // strip, and strips up to nine compute warps wide (a domain that fits
        // one strip wraps in shared memory)
        const std::vector<int> bxs =
            h->descs[0].compact ? std::vector<int>{32, 64, 96, 128, 160, 192, 224, 256, 288}
                                : std::vector<int>{64, 128, 256};
        const int rws[] = {4, 8, 16, 32, 64, 128};
        for (int bx : bxs)
            for (int r : rws) {
                if (r > max_ny && r != rws[0]) continue;
                lb_schedule s = h->sched;
                s.n_class = 1;
                s.block_x[0] = bx;
                s.rows[0] = r;
                cands.push_back(s);
            }
    }
    cudaEvent_t e0, e1;
    LB_CUDA(cudaEventCreate(&e0));
    LB_CUDA(cudaEventCreate(&e1));
    const lb_schedule old = h->sched;
    double best = 1e300;
    lb_schedule chosen = old;
    int rc = LB_OK;
    // one timing of a candidate (ms per step); negative on failure
    auto time_candidate = [&](const lb_schedule& c, int len, int r) -> double {
        if ((rc = lb_set_schedule(h, &c)) != LB_OK) return -1.0;
        if (h->n_dom > 1 || !plain) return time_graph_steps(h, len, r, e0, e1);
        // warm-up, then time `r` launches that read the current buffer and
        // write the idle one (the state itself does not advance)
        if ((rc = enqueue_step(h, h->parity, h->stream)) != LB_OK) return -1.0;
        cudaEventRecord(e0, h->stream);
        for (int k = 0; k < r && rc == LB_OK; ++k) rc = enqueue_step(h, h->parity, h->stream);
        cudaEventRecord(e1, h->stream);
        if (rc != LB_OK) return -1.0;
        float t = 0.f;
        h->launches += (r + 1) * launches_per_step(h);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return -1.0;
        return double(t) / r;
    };
    // a batch: graphs of 16 steps, so that chains and tails show; then the
    // fastest eight again over graphs of the length the steps run in (the
    // leading candidates are within a few percent of each other)
    std::vector<std::pair<double, size_t>> scored;
    for (size_t k = 0; k < cands.size(); ++k) {
        const double ms = time_candidate(cands[k], h->n_dom > 1 || !plain ? 16 : 4, reps);
        if (ms < 0.0) {
            if (rc == LB_OK) rc = LB_ERR_CUDA;
            break;
        }
        scored.emplace_back(ms, k);
    }
    if (rc == LB_OK && (h->n_dom > 1 || !plain) && scored.size() > 1) {
        std::sort(scored.begin(), scored.end());
        const size_t top = std::min<size_t>(8, scored.size());
        for (size_t t = 0; t < top && rc == LB_OK; ++t) {
            const double ms = time_candidate(cands[scored[t].second], kGraphBig, reps + 3);
            if (ms < 0.0) {
                if (rc == LB_OK) rc = LB_ERR_CUDA;
                break;
            }
            scored[t].first = ms;
        }
        scored.resize(top);
    }
    for (const auto& sc : scored)
        if (sc.first < best) {
            best = sc.first;
            chosen = cands[sc.second];
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == LB_OK) rc = sync_and_check(h);
    const int rc2 = lb_set_schedule(h, rc == LB_OK ? &chosen : &old);
    if (rc != LB_OK) return rc;
    if (rc2 != LB_OK) return rc2;
    if (block_x) *block_x = h->block_x();
    if (rows) *rows = h->rows();
    if (best_ms) *best_ms = best;
    return LB_OK;
}

long long lb_step_count(const lb_handle* h) { return h ? h->steps : -1; }

int lb_sync(lb_handle* h)
{
    if (use_device(h) != LB_OK) return h ? LB_ERR_CUDA : LB_ERR_INVALID_ARG;
    return sync_and_check(h);
}

long long lb_launch_count(const lb_handle* h) { return h ? h->launches : -1; }

int lb_check_wait_timeout(void* stream)
{
    unsigned word = 0;
    const int e = lbfe::run_wait_selfcheck(stream, &word);
    if (e != 0) return fail(LB_ERR_CUDA, "self-check launch failed: %s", cudaGetErrorString(cudaError_t(e)));
    if (word == 3u) return fail(LB_ERR_TIMEOUT, "bounded waits gave up as designed (word 0x%x)", word);
    return fail(LB_OK, "a bounded wait did not give up (word 0x%x)", word);
}

const char* lb_error_string(int code)
{
    switch (code) {
        case LB_OK: return "ok";
        case LB_ERR_INVALID_ARG: return "invalid argument";
        case LB_ERR_CUDA: return "CUDA error";
        case LB_ERR_NONFINITE: return "non-finite state";
        case LB_ERR_TIMEOUT: return "device wait timed out";
        case LB_ERR_NO_INTERFACE: return "no interface to fit";
        case LB_ERR_CAPACITY: return "interface buffer too small";
        default: return "unknown error";
    }
}

const char* lb_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
