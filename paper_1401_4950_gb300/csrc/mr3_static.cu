// mr3_static.cu -- mr3_stemr_static: the one-matrix solve of mr3_stemr with every byte of
// device workspace taken from one file-scope device array, so that a call allocates no
// device memory.  The kernels are the ones mr3_stemr launches; only the host driver differs:
// it carves its buffers out of the array and runs every step on the caller's stream, one
// after the other (no side stream, no events).
//
// Who needs this: mr3_stemr draws its workspace from the stream-ordered memory pool.  A
// process whose device memory is claimed in full by its own caching allocator when it
// starts (a serving process sizing its key-value cache to the card, for instance) has no
// room for the pool to grow into, and a caller inside a latency-critical loop may not be
// allowed to enter an allocator at all.  Such callers get a solver with a fixed footprint
// here: the array below, reserved when this translation unit's module is loaded.
//
// Set-up: on the first call made with a given device current (any order n up to the
// limit, n = 0 included), the library loads, on that device, every kernel this entry point
// launches and the array itself, and looks up the address of that device's copy of the
// array once (cudaGetSymbolAddress) and caches it; later calls reuse it.  The runtime
// otherwise loads each kernel at its first launch, and loading takes device memory.  So a
// caller that claims its device memory up front should make one call per device (n = 0
// is enough) before doing so, and the first call on each device should come before the
// caller begins any stream capture.  None of these kernels uses a stack frame, so no
// launch grows the device's local-memory reservation.
//
// Sharing: each device has exactly one array.  Two calls that overlap in time on the same
// device (two host threads, or two streams not ordered with respect to each other) write
// the same bytes and race; the caller must order them.
#include <algorithm>
#include <cstring>
#include <mutex>
#include "mr3.h"
#include "mr3_kernels.h"

namespace mr3 {
namespace {

__device__ __align__(256) unsigned char g_static_scratch[MR3_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the current device's array (looked up on the first call per device).
int static_scratch(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MR3_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return MR3_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p ||
            preload_prologue() != cudaSuccess || preload_levels() != cudaSuccess ||
            preload_rqi() != cudaSuccess) {
            cudaGetLastError();
            return MR3_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return 0;
}

// Two-ended bump allocator over the array.  Buffers that live for the whole call are
// taken from the low end first (then `fixed` marks their top).  The representation tree
// alternates ends by level: the buffers of level L+1 go to end (L+1) & 1, which first
// drops what level L-1 left there; everything runs in order on one stream, so every
// kernel reading level L-1 was enqueued before anything can overwrite it.
struct Arena {
    char *base;
    size_t size;
    size_t lo = 0, hi;
    size_t fixed = 0;
    bool full = false;
    Arena(void *p, size_t bytes) : base((char *)p), size(bytes), hi(bytes) {}
    static size_t round_up(size_t b) { return (b + 255) & ~(size_t)255; }
    template <class T> T *take(size_t count, int end) {
        const size_t b = round_up(std::max<size_t>(count, 1) * sizeof(T));
        if (b > hi - lo) {
            full = true;
            return nullptr;
        }
        if (end == 0) {
            T *p = (T *)(base + lo);
            lo += b;
            return p;
        }
        hi -= b;
        return (T *)(base + hi);
    }
    template <class T> T *low(size_t count) { return take<T>(count, 0); }
    void seal_fixed() { fixed = lo; }
    void reset_end(int end) {
        if (end == 0) lo = fixed;
        else hi = size;
    }
};

#define SCK(call)                                                                        \
    do {                                                                                 \
        if ((call) != cudaSuccess) {                                                     \
            cudaGetLastError();                                                          \
            return MR3_ECUDA;                                                            \
        }                                                                                \
    } while (0)
#define SFULL(ar)                                                                        \
    do {                                                                                 \
        if ((ar).full) return MR3_ENOSCRATCH;                                            \
    } while (0)

int lanes_auto(long long nactive, int tpe, int warps_per_sm) {
    return bisect_lanes(nactive, warps_per_sm, tpe);
}

// The solve of one matrix (M filled in by the entry point) on the array behind `ar`.
int solve_static(MatDesc &M, const double *d, const double *e, int range, double *w, double *Z,
                 const mr3_opts *opts, mr3_info &out, Arena &ar, cudaStream_t s) {
    const double gaptol = (opts && opts->gaptol > 0.0) ? opts->gaptol : kGaptolAuto;
    const unsigned long long seed = (opts && opts->seed) ? opts->seed : 0x5EEDull;
    const int max_rqi = (opts && opts->max_rqi > 0) ? opts->max_rqi : 10;
    const int max_tries = (opts && opts->max_shift_tries > 0) ? opts->max_shift_tries : 8;
    const unsigned fault_mask = opts ? opts->fault_mask : 0u;
    const int tpe = opts ? opts->tpe : 0;
    const int bwarps = (opts && opts->bisect_warps > 0 && opts->bisect_warps <= 64) ? opts->bisect_warps : 48;
    const int max_depth = (opts && opts->max_depth > 0) ? opts->max_depth : 64;
    // the absolute-gap split is not taken here: the array holds the root's clusters on the
    // assumption that each has two members or more
    const int erep = (opts && opts->erep) ? 1 : 0;
    const long long n = M.n;

    MatDesc *dmats = ar.low<MatDesc>(1);
    DevInfo *dinfo = ar.low<DevInfo>(1);
    int *dint = ar.low<int>(4);
    int *flags = ar.low<int>(n);
    int *scanned = ar.low<int>(n);
    int *scan_tmp = ar.low<int>(scan_tmp_ints(n));
    SFULL(ar);
    // the array keeps whatever the previous call left: clear every accumulator
    SCK(cudaMemcpyAsync(dmats, &M, sizeof(MatDesc), cudaMemcpyHostToDevice, s));
    SCK(cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s));
    SCK(cudaMemsetAsync(dint, 0, 4 * sizeof(int), s));
    launch_mat_norm(1, dmats, d, e, dint, s);
    launch_split_flags(1, dmats, n, d, e, flags, s);
    launch_exclusive_scan(flags, scanned, n, dint + 1, scan_tmp, s);
    int hint[4];
    SCK(cudaMemcpyAsync(hint, dint, sizeof(hint), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (hint[0]) {
        M.m = 0;
        out.status_counts[MR3_SNONFINITE] = 1;
        return MR3_SNONFINITE;
    }
    const int nblk = hint[1];
    BlkDesc *blks = ar.low<BlkDesc>(nblk);
    SFULL(ar);
    build_blocks(n, flags, scanned, dint + 1, nblk, 1, dmats, blks, s);
    launch_blk_setup(nblk, blks, 1, dmats, d, e, range, s);
    if (range == MR3_RANGE_INDEX) launch_index_multi(1, dmats, blks, d, e, s);
    launch_assign_columns(1, dmats, blks, range, s);
    SCK(cudaMemcpyAsync(&M, dmats, sizeof(MatDesc), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    const long long mtotal = M.m;
    out.nblocks = nblk;
    out.m = M.m;
    if (mtotal == 0) return 0;

    // ---- root representations and level-0 intervals
    const long long ncols = n;
    double *pool0 = ar.low<double>((size_t)kRepStride * n + (size_t)kRepPad * nblk);
    int *grid = ar.low<int>(ncols + 64ll * nblk + 1);
    float *f32 = ar.low<float>(2 * n);
    Node *nodes0 = ar.low<Node>(nblk);
    int *cnode = ar.low<int>(ncols);
    int *jloc = ar.low<int>(ncols);
    double *lo = ar.low<double>(ncols);
    double *hi = ar.low<double>(ncols);
    double *gapl = ar.low<double>(ncols);
    double *gapr = ar.low<double>(ncols);
    SingleItem *singles = ar.low<SingleItem>(ncols);
    ClusterItem *clusters = ar.low<ClusterItem>(ncols / 2 + 1);
    long long *crep = ar.low<long long>(ncols / 2 + 1);
    LevelCounters *ctr = ar.low<LevelCounters>(1);
    int *work = ar.low<int>(1);
    // RQI scratch: up to a quarter of the array, at most one warp slot per 4 singletons
    // lanes per singleton: 8, the latency-bound choice for one matrix and the instance
    // compiled without a stack frame (opts->rqi_team is not applied here)
    const int team = 8;
    const size_t slot_bytes = (size_t)rqi_scratch_per_index(team) * n * sizeof(double);
    const long long want_slots = (mtotal + rqi_singles_per_slot(team) - 1) / rqi_singles_per_slot(team);
    const long long cap_slots = std::max<long long>(1, (MR3_STATIC_SCRATCH_BYTES / 4) / slot_bytes);
    const int slots = (int)std::min(want_slots, cap_slots);
    double *rqi_scratch = ar.low<double>((size_t)slots * rqi_scratch_per_index(team) * n);
    SFULL(ar);
    ar.seal_fixed();
    SCK(cudaMemsetAsync(cnode, 0xff, sizeof(int) * ncols, s));
    launch_root(nblk, blks, d, e, pool0, f32, seed, s);
    launch_init_columns(nblk, blks, nodes0, cnode, jloc, lo, hi, (int)ncols, s);
    const double rtol = 1e-2 * (gaptol > 0.0 ? gaptol : 1e-3);
    if (range != MR3_RANGE_ALL) launch_outer_gaps(nblk, blks, nodes0, pool0, rtol, dinfo, s);
    if (M.nblk > 1) launch_zero_z(1, dmats, Z, s);
    launch_grid(nblk, blks, nodes0, pool0, grid, lo, hi, M.m, dinfo, s);
    launch_bisect((int)ncols, nullptr, lanes_auto(mtotal, tpe, bwarps), (int)ncols, cnode, nodes0, blks,
                  pool0, jloc, lo, hi, rtol, nullptr, dinfo, s);

    // ---- level loop, all on stream s: classify; singletons by RQI; clusters shifted and
    // refined on their child representations.
    Node *cur_nodes = nodes0;
    double *cur_pool = pool0;
    int ncur = nblk;
    int status = 0;
    for (int level = 0;; ++level) {
        SCK(cudaMemsetAsync(ctr, 0, sizeof(LevelCounters), s));
        launch_classify(ncur, cur_nodes, blks, lo, hi, gaptol, 0.0, gapl, gapr, singles, clusters,
                        crep, cnode, ctr, dinfo, s);
        LevelCounters hc;
        SCK(cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
        SCK(cudaStreamSynchronize(s));
        if (hc.nsingle > 0)
            launch_rqi(hc.nsingle, singles, cur_nodes, blks, dmats, cur_pool, jloc, lo, hi, gapl,
                       gapr, d, e, w, Z, rqi_scratch, slots, (int)n, max_rqi, fault_mask, work,
                       dinfo, team, s);
        if (hc.ncluster == 0) break;
        const int end = (level + 1) & 1;
        ar.reset_end(end);
        double *next_pool = ar.take<double>((size_t)hc.pool_need, end);
        Node *next_nodes = ar.take<Node>(hc.ncluster, end);
        double *tau = ar.take<double>(hc.ncluster, end);
        int *next_active = ar.take<int>(hc.nactive, end);
        double2 *tri = ar.take<double2>(2 * (size_t)hc.ncluster, end);
        char *shift_ws = ar.take<char>(shift_scratch_bytes(hc.ncluster, max_tries), end);
        SFULL(ar);
        launch_refine_ends(hc.ncluster, clusters, cur_nodes, blks, cur_pool, jloc, lo, hi, tri, dinfo, s);
        launch_shift(hc.ncluster, clusters, crep, cur_nodes, blks, cur_pool, next_pool, next_nodes,
                     tau, cnode, next_active, jloc, lo, hi, max_tries, fault_mask, erep, tri,
                     shift_ws, dinfo, s);
        launch_bisect(hc.nactive, next_active, lanes_auto(hc.nactive, tpe, bwarps), (int)ncols, cnode,
                      next_nodes, blks, next_pool, jloc, lo, hi, rtol, tau, dinfo, s);
        cur_pool = next_pool;
        cur_nodes = next_nodes;
        ncur = hc.ncluster;
        if (level + 1 >= max_depth) {
            // depth cap: the remaining members are finished as singletons (flagged)
            status = MR3_SDEPTH;
            SCK(cudaMemsetAsync(ctr, 0, sizeof(LevelCounters), s));
            launch_classify(ncur, cur_nodes, blks, lo, hi, -1e308, 0.0, gapl, gapr, singles, clusters,
                            crep, cnode, ctr, dinfo, s);
            SCK(cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
            SCK(cudaStreamSynchronize(s));
            if (hc.nsingle > 0)
                launch_rqi(hc.nsingle, singles, cur_nodes, blks, dmats, cur_pool, jloc, lo, hi,
                           gapl, gapr, d, e, w, Z, rqi_scratch, slots, (int)n, max_rqi,
                           fault_mask, work, dinfo, team, s);
            break;
        }
    }

    // ---- ascending output order (the tree's buffers are dead: reuse both ends)
    ar.reset_end(0);
    ar.reset_end(1);
    int *oflag = ar.low<int>(1);
    SFULL(ar);
    launch_order_flags(1, dmats, w, oflag, s);
    int hflag = 0;
    SCK(cudaMemcpyAsync(&hflag, oflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (hflag && M.m > 1) {
        double *wtmp = ar.low<double>(M.m);
        double *ztmp = ar.low<double>((size_t)M.m * M.n);
        int *perm = ar.low<int>(M.m);
        SFULL(ar);
        launch_sort_outputs(0, M.m, dmats, w, Z, wtmp, ztmp, perm, s);
    }
    DevInfo h;
    SCK(cudaMemcpyAsync(&h, dinfo, sizeof(h), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    SCK(cudaGetLastError());
    out.dmax = h.dmax;
    out.nclusters = h.nclusters;
    out.largest_cluster = h.largest;
    out.new_rrr = h.new_rrr;
    out.untested_rrr = h.untested;
    out.rqi_iters = (long long)h.rqi_iters;
    out.rqi_iters_max = h.rqi_max;
    out.bisect_fallbacks = h.fallbacks;
    out.sturm_steps = (long long)h.sturm_steps;
    out.shift_steps = (long long)h.shift_steps;
    out.twisted_steps = (long long)h.twisted_steps;
    out.ladder_clusters = h.ladder;
    out.recomputed_rrr = h.recomputed;
    out.envelope_rrr = h.env_accepted;
    for (int k = 0; k < 8; ++k) out.status_counts[k] = h.status[k];
    if (status) {
        out.status_counts[status] += 1;
        return status;
    }
    if (h.status[MR3_SCAP]) return MR3_SCAP;
    if (h.status[MR3_SUNTESTED_RRR]) return MR3_SUNTESTED_RRR;
    return 0;
}

} // namespace
} // namespace mr3

using namespace mr3;

extern "C" int mr3_stemr_static(int n, const double *d, const double *e, int range, double vl,
                                double vu, int il, int iu, int *m, double *w, double *Z, int ldz,
                                const mr3_opts *opts, mr3_info *info, void *stream) {
    if (n < 0) return -1;
    if (n > 0 && !d) return -2;
    if (n > 1 && !e) return -3;
    if (range < MR3_RANGE_ALL || range > MR3_RANGE_INDEX) return -4;
    if (range == MR3_RANGE_VALUE && !(vl < vu)) return -6;
    if (range == MR3_RANGE_INDEX) {
        if (n == 0) { if (!(il == 1 && iu == 0)) return -7; }
        else {
            if (il < 1 || il > n) return -7;
            if (iu < il || iu > n) return -8;
        }
    }
    if (!m) return -9;
    if (n > 0 && !w) return -10;
    if (n > 0 && !Z) return -11;
    if (ldz < std::max(1, n)) return -12;
    if (opts && opts->prec == MR3_DD) return -13; // the binary64 tree only
    *m = 0;
    mr3_info out;
    std::memset(&out, 0, sizeof(out));
    if (n > MR3_STATIC_MAX_N) {
        if (info) *info = out;
        return MR3_ENOSCRATCH;
    }
    void *base = nullptr;
    const int src = static_scratch(&base); // set-up on the first call per device
    if (src) {
        if (info) *info = out;
        return src;
    }
    if (n == 0) {
        if (info) *info = out;
        return 0;
    }
    MatDesc M;
    std::memset(&M, 0, sizeof(M));
    M.n = n;
    M.ldz = ldz;
    M.il = il;
    M.iu = iu;
    M.vl = vl;
    M.vu = vu;
    Arena ar(base, MR3_STATIC_SCRATCH_BYTES);
    const int rc = solve_static(M, d, e, range, w, Z, opts, out, ar, (cudaStream_t)stream);
    if (rc == MR3_ENOSCRATCH || rc == MR3_ECUDA) {
        cudaStreamSynchronize((cudaStream_t)stream); // nothing enqueued may outlive the call
        cudaGetLastError();
        std::memset(&out, 0, sizeof(out));
        if (info) *info = out;
        return rc;
    }
    *m = M.m;
    if (info) *info = out;
    return rc;
}
