// mr3_api.cu -- C ABI entry points and the host side of the solver: argument checks,
// workspace, and the level-by-level traversal of the representation tree (Alg. MRRR,
// breadth first: per level classify, singletons by RQI, clusters by a shift and a
// refinement on the child representation).
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>
#include "mr3.h"
#include "mr3_kernels.h"

namespace mr3 {

// Bisection lanes per eigenvalue keep about this many warps per SM in flight by default.
#ifndef MR3_BISECT_WARPS_PER_SM
#define MR3_BISECT_WARPS_PER_SM 48
#endif

namespace {

struct Opts {
    int prec;
    double gaptol;
    unsigned long long seed;
    int max_rqi;
    int max_tries;
    unsigned fault_mask;
    int tpe;
    int max_depth;
    int profile;
    int rqi_team;
    int bisect_warps;
    int abs_split;
    int erep;
    int graph;
};

Opts resolve(const mr3_opts *o) {
    Opts r;
    r.prec = (o && o->prec == MR3_DD) ? MR3_DD : MR3_FP64;
    r.gaptol = (o && o->gaptol > 0.0) ? o->gaptol : (r.prec == MR3_DD ? 1e-10 : kGaptolAuto);
    r.seed = (o && o->seed) ? o->seed : 0x5EEDull;
    r.max_rqi = (o && o->max_rqi > 0) ? o->max_rqi : 10;
    r.max_tries = (o && o->max_shift_tries > 0) ? o->max_shift_tries : 8;
    r.fault_mask = o ? o->fault_mask : 0u;
    r.tpe = o ? o->tpe : 0;
    r.max_depth = (o && o->max_depth > 0) ? o->max_depth : 64;
    r.profile = o ? o->profile : 0;
    r.rqi_team = (o && (o->rqi_team == 2 || o->rqi_team == 8)) ? o->rqi_team : 0;
    r.bisect_warps = (o && o->bisect_warps > 0 && o->bisect_warps <= 64) ? o->bisect_warps
                                                                         : MR3_BISECT_WARPS_PER_SM;
    r.abs_split = (o && o->abs_split > 0) ? 1 : 0;
    r.erep = (o && o->erep) ? 1 : 0;
    r.graph = o ? (o->graph > 0 ? 1 : (o->graph < 0 ? -1 : 0)) : 0;
    return r;
}

// Lanes per eigenvalue for the multisection: enough lanes in flight to keep the SMs busy
// (about MR3_BISECT_WARPS_PER_SM warps per SM on 152 SMs), at most 32; opts->tpe overrides.
// Levels unrolled in the graph-captured level loop, and the number of matrices from which a
// solve takes that loop by default (opts->graph = 0).
#ifndef MR3_GRAPH_LEVELS
#define MR3_GRAPH_LEVELS 12
#endif
constexpr int kGraphLevels = MR3_GRAPH_LEVELS;
constexpr int kGraphMinMatrices = 2;

int lanes_for(long long nactive, const Opts &o) {
    return bisect_lanes(nactive, o.bisect_warps, o.tpe);
}

// Warp slots (one warp each) for an RQI launch with the given team size: one per
// rqi_singles_per_slot(team) singletons, within a scratch budget of cap_bytes.
long long rqi_slots(long long nsingle, int nmax, long long cap_bytes, int team) {
    const int per = rqi_singles_per_slot(team);
    const long long want = (nsingle + per - 1) / per;
    const long long per_slot = (long long)rqi_scratch_per_index(team) * nmax * (long long)sizeof(double);
    const long long cap = std::max<long long>(152, cap_bytes / per_slot);
    return std::min(want, cap);
}

// Optional per-group device timing: an event pair around every launch group, on the
// call's stream; durations are read after the final synchronisation.
struct Prof {
    bool on;
    cudaStream_t s;
    std::vector<cudaEvent_t> evs;
    std::vector<int> group;
    std::vector<int> nlaunch;
    explicit Prof(bool enabled, cudaStream_t st) : on(enabled), s(st) {}
    int begin(cudaStream_t st = nullptr) {
        if (!on) return -1;
        cudaEvent_t a;
        cudaEventCreate(&a);
        cudaEventRecord(a, st ? st : s);
        evs.push_back(a);
        return (int)evs.size() - 1;
    }
    void end(int tok, int g, int launches, cudaStream_t st = nullptr) {
        if (!on || tok < 0) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, st ? st : s);
        evs.push_back(b);
        group.push_back(g);
        nlaunch.push_back(launches);
    }
    void collect(mr3_info &out) {
        if (!on) return;
        for (size_t k = 0; k < group.size(); ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, evs[2 * k], evs[2 * k + 1]);
            out.kernel_ms[group[k]] += ms;
            out.kernel_launches[group[k]] += nlaunch[k];
        }
    }
    ~Prof() {
        for (auto e : evs) cudaEventDestroy(e);
    }
};

// MR3_TRACE set (and not "0") in the environment: the host-driven level loop prints one
// line per tree level on stderr: singletons, clusters, the largest cluster, the columns to
// refine, the stream times of the level's cluster-end refinement, shift and child
// bisection (event pairs on the main stream; the singletons run beside them), and the
// sweep statistics of its multisection launches.  Diagnostic only: it synchronises the
// stream once per level.
bool trace_on() {
    static const bool v = [] {
        const char *t = std::getenv("MR3_TRACE");
        return t && *t && std::strcmp(t, "0") != 0;
    }();
    return v;
}

struct TraceLevel {
    int level;
    LevelCounters hc;
    cudaEvent_t ev[4];
    DevInfo sweeps; // the multisection statistics of the level's launches
};
struct TraceLog : std::vector<TraceLevel> {
    ~TraceLog() {
        for (auto &t : *this)
            for (auto ev : t.ev)
                if (ev) cudaEventDestroy(ev);
    }
};

} // namespace

// ------------------------------------------------------------------ memory pool

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxDevices] = {};
} // namespace

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        pool = g_pools[dev];
        if (!pool) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
                cudaGetLastError();
                return cudaMallocAsync(p, bytes, s);
            }
            unsigned long long keep = ~0ull; // never trimmed at synchronisation
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            g_pools[dev] = pool;
        }
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// ------------------------------------------------------------------ counter read-back

namespace {

// Counters the host reads between launches (the level's singleton and cluster counts, the
// matrix descriptors, the statistics) travel without a copy engine: a small kernel stores
// them into mapped pinned host memory, and the host reads them once the stream has
// synchronised.  A cudaMemcpyAsync to the host would queue behind any large transfer the
// caller has in flight on the same copy engine (a 1.6 GB read of a previous result held
// every tree level's read for its full duration).  One growing buffer per host thread;
// with unified addressing its host address is also its device address.
struct MappedBuffer {
    void *h = nullptr;
    size_t bytes = 0;
};
thread_local MappedBuffer t_mapped;

__global__ void k_publish(const unsigned *__restrict__ src, unsigned *dst, size_t words) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

} // namespace

// Copies bytes (a multiple of 4) from device memory to host memory in stream order and
// waits for them.
cudaError_t read_back(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    if (bytes % 4 != 0) {
        cudaError_t err = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
        return err != cudaSuccess ? err : cudaStreamSynchronize(s);
    }
    if (t_mapped.bytes < bytes) {
        if (t_mapped.h) cudaFreeHost(t_mapped.h);
        t_mapped = MappedBuffer();
        const size_t want = std::max<size_t>(bytes, 64 << 10);
        void *h = nullptr;
        cudaError_t err = cudaHostAlloc(&h, want, cudaHostAllocMapped | cudaHostAllocPortable);
        if (err != cudaSuccess) return err;
        t_mapped.h = h;
        t_mapped.bytes = want;
    }
    void *dptr = nullptr;
    cudaError_t err = cudaHostGetDevicePointer(&dptr, t_mapped.h, 0);
    if (err != cudaSuccess) return err;
    const size_t words = bytes / 4;
    const unsigned blocks = (unsigned)std::min<size_t>((words + 255) / 256, 64);
    k_publish<<<blocks, 256, 0, s>>>((const unsigned *)src, (unsigned *)dptr, words);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    memcpy(dst, t_mapped.h, bytes);
    return cudaSuccess;
}

namespace {

// Stream-ordered workspace: every block is returned (cudaFreeAsync) when the call ends.
struct Workspace {
    cudaStream_t s;
    std::vector<void *> blocks;
    bool oom = false;
    explicit Workspace(cudaStream_t st) : s(st) {}
    template <class T> T *get(size_t count) {
        void *p = nullptr;
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        if (lib_malloc_async(&p, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            oom = true;
            return nullptr;
        }
        blocks.push_back(p);
        return (T *)p;
    }
    void release(void *p) {
        if (!p) return;
        auto it = std::find(blocks.begin(), blocks.end(), p);
        if (it != blocks.end()) {
            cudaFreeAsync(p, s);
            blocks.erase(it);
        }
    }
    ~Workspace() {
        for (void *p : blocks) cudaFreeAsync(p, s);
    }
};

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            cudaGetLastError();                                                          \
            return (e_ == cudaErrorMemoryAllocation) ? MR3_EOOM : MR3_ECUDA;             \
        }                                                                                \
    } while (0)
#define CKW(ws)                                                                          \
    do {                                                                                 \
        if ((ws).oom) return MR3_EOOM;                                                   \
    } while (0)

// The solver proper, for nmat matrices described by host MatDesc entries (off, n, zoff,
// ldz, woff and the range data filled in).  ncols: size of the global column space.
// On return mats[b].m holds the eigenpairs of matrix b.
int solve(int nmat, std::vector<MatDesc> &mats, long long nrows, long long ncols,
          const double *d, const double *e, int range, double *w, double *Z, const Opts &o,
          mr3_info *info, cudaStream_t s) {
    Workspace ws(s);
    mr3_info out;
    std::memset(&out, 0, sizeof(out));
    if (nrows == 0 || nmat == 0) {
        for (auto &M : mats) M.m = 0;
        if (info) *info = out;
        return 0;
    }
    MatDesc *dmats = ws.get<MatDesc>(nmat);
    DevInfo *dinfo = ws.get<DevInfo>(1);
    int *dint = ws.get<int>(4); // [0] bad input, [1] number of blocks
    int *flags = ws.get<int>(nrows);
    int *scanned = ws.get<int>(nrows);
    int *scan_tmp = ws.get<int>(scan_tmp_ints(nrows));
    CKW(ws);
    CK(cudaMemcpyAsync(dmats, mats.data(), sizeof(MatDesc) * nmat, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dinfo, 0, sizeof(DevInfo), s));
    CK(cudaMemsetAsync(dint, 0, 4 * sizeof(int), s));
    Prof prof(o.profile != 0, s);
    int tk = prof.begin();
    launch_mat_norm(nmat, dmats, d, e, dint, s);
    launch_split_flags(nmat, dmats, nrows, d, e, flags, s);
    launch_exclusive_scan(flags, scanned, nrows, dint + 1, scan_tmp, s);
    prof.end(tk, 0, 5);
    int hint[4];
    CK(read_back(hint, dint, sizeof(hint), s));
    if (hint[0]) {
        for (auto &M : mats) M.m = 0;
        out.status_counts[MR3_SNONFINITE] = 1;
        if (info) *info = out;
        return MR3_SNONFINITE;
    }
    const int nblk = hint[1];
    BlkDesc *blks = ws.get<BlkDesc>(nblk);
    CKW(ws);
    tk = prof.begin();
    build_blocks(nrows, flags, scanned, dint + 1, nblk, nmat, dmats, blks, s);
    launch_blk_setup(nblk, blks, nmat, dmats, d, e, range, s);
    if (range == MR3_RANGE_INDEX) launch_index_multi(nmat, dmats, blks, d, e, s);
    launch_assign_columns(nmat, dmats, blks, range, s);
    prof.end(tk, 0, range == MR3_RANGE_INDEX ? 6 : 5);
    CK(read_back(mats.data(), dmats, sizeof(MatDesc) * nmat, s));
    ws.release(flags);
    ws.release(scanned);
    ws.release(scan_tmp);
    long long mtotal = 0;
    int nmax = 1;
    for (auto &M : mats) { mtotal += M.m; nmax = std::max(nmax, M.n); }
    out.nblocks = nblk;
    out.m = (int)std::min<long long>(mtotal, 0x7fffffff);
    if (mtotal == 0) {
        if (info) *info = out;
        return 0;
    }
    // ---- root representations and level-0 intervals.  With the double-double tree a
    // pool holds a second plane of low-order words right behind the leading ones.
    const bool dd = (o.prec == MR3_DD);
    const size_t pool0_len = (size_t)kRepStride * nrows + (size_t)kRepPad * nblk;
    double *pool0 = ws.get<double>(dd ? 2 * pool0_len : pool0_len);
    double *pool0_lo = dd && pool0 ? pool0 + pool0_len : nullptr;
    int *grid = ws.get<int>(ncols + 64ll * nblk + 1);
    float *f32 = ws.get<float>(2 * nrows);
    Node *nodes0 = ws.get<Node>(nblk);
    int *cnode = ws.get<int>(ncols);
    int *jloc = ws.get<int>(ncols);
    double *lo = ws.get<double>(ncols);
    double *hi = ws.get<double>(ncols);
    double *gapl = ws.get<double>(ncols);
    double *gapr = ws.get<double>(ncols);
    SingleItem *singles = ws.get<SingleItem>(ncols);
    // clusters have two members or more, except the root's pieces of the absolute-gap split
    const long long max_clusters = o.abs_split ? ncols + 1 : ncols / 2 + 1;
    ClusterItem *clusters = ws.get<ClusterItem>(max_clusters);
    long long *crep = ws.get<long long>(max_clusters);
    LevelCounters *ctr = ws.get<LevelCounters>(1);
    int *work = ws.get<int>(1);
    CKW(ws);
    CK(cudaMemsetAsync(cnode, 0xff, sizeof(int) * ncols, s));
    tk = prof.begin();
    launch_root(nblk, blks, d, e, pool0, f32, o.seed, s);
    if (dd) launch_root_dd(nblk, blks, d, e, pool0, pool0_lo, o.seed, s);
    launch_init_columns(nblk, blks, nodes0, cnode, jloc, lo, hi, (int)ncols, s);
    prof.end(tk, 1, dd ? 3 : 2);
    // classification accuracy (Sec. 3.2.2): 1e-2 gaptol, with the smallest automatic
    // gaptol (1e-3) standing in for the per-block choice
    const double rtol = 1e-2 * (o.gaptol > 0.0 ? o.gaptol : 1e-3);
    if (range != MR3_RANGE_ALL) launch_outer_gaps(nblk, blks, nodes0, pool0, rtol, dinfo, s);
    bool any_multi = false;
    for (auto &M : mats) any_multi |= (M.nblk > 1 && M.m > 0);
    if (any_multi) launch_zero_z(nmat, dmats, Z, s);
    tk = prof.begin();
    {
        int max_m = 0;
        for (auto &M : mats) max_m = std::max(max_m, M.m);
        launch_grid(nblk, blks, nodes0, pool0, grid, lo, hi, max_m, dinfo, s);
        launch_bisect((int)ncols, nullptr, lanes_for(mtotal, o), (int)ncols, cnode, nodes0, blks,
                      pool0, jloc, lo, hi, rtol, nullptr, dinfo, s);
    }
    prof.end(tk, 2, 3);
    ws.release(f32);

    // ---- level loop.  The singletons of a level are finished by RQI on a side stream
    // (ordered after that level's classification by an event) while the main stream goes
    // on with the level's clusters; the two touch disjoint columns.  The singleton list is
    // double-buffered, and a level's representation pool is returned only after its RQI.
    cudaStream_t side = nullptr;
    CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    struct SideGuard {
        cudaStream_t st;
        std::vector<cudaEvent_t> evs;
        ~SideGuard() {
            if (st) cudaStreamSynchronize(st);
            for (auto e : evs) cudaEventDestroy(e);
            if (st) cudaStreamDestroy(st);
        }
        cudaEvent_t make() {
            cudaEvent_t e;
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            evs.push_back(e);
            return e;
        }
    } guard{side, {}};
    SingleItem *singles2[2] = {singles, ws.get<SingleItem>(ncols)};
    CKW(ws);
    struct Pending { double *pool; Node *nodes; cudaEvent_t done; };
    std::vector<Pending> pending;   // pools/nodes still read by an RQI launch
    std::vector<cudaEvent_t> rqi_done(2, nullptr);
    Node *cur_nodes = nodes0;
    double *cur_pool = pool0, *cur_lo = pool0_lo;
    int ncur = nblk;
    double *scratch = nullptr;
    size_t scratch_len = 0; // doubles
    // RQI scratch budget per launch: enough for every root-level singleton of a few
    // n = 8192 matrices to run at once with teams of 2 (~10 warps per SM), where the
    // latency of the scratch and representation loads is hidden by other warps; the slot
    // count is halved while the allocation fails
    const long long scratch_cap_bytes = 8ll << 30;
    int status = 0;
    auto run_singles = [&](int level, const LevelCounters &hc) -> int {
        const int team = dd ? 0 : (o.rqi_team ? o.rqi_team : rqi_team(hc.nsingle, nmat));
        long long slots = dd ? rqi_dd_threads(hc.nsingle, nmax, 2 * scratch_cap_bytes)
                             : rqi_slots(hc.nsingle, nmax, scratch_cap_bytes, team);
        const size_t per_slot = dd ? (size_t)4 * nmax : (size_t)rqi_scratch_per_index(team) * nmax;
        if ((size_t)slots * per_slot > scratch_len) {
            if (scratch) cudaFreeAsync(scratch, side); // after the side stream's last use
            scratch = nullptr;
            scratch_len = 0;
            for (;;) {
                const size_t need = (size_t)slots * per_slot;
                void *p = nullptr;
                if (lib_malloc_async(&p, need * sizeof(double), s) == cudaSuccess) {
                    scratch = (double *)p;
                    scratch_len = need;
                    break;
                }
                cudaGetLastError();
                // binary64 teams: at least one warp per SM; double-double: whole blocks of 128
                const long long minslots = dd ? 128 : 152;
                if (slots <= minslots) return MR3_EOOM;
                slots = std::max<long long>(minslots, dd ? (slots / 2) / 128 * 128 : slots / 2);
            }
        }
        cudaEvent_t ready = guard.make();
        cudaEventRecord(ready, s);
        cudaStreamWaitEvent(side, ready, 0);
        const int tq = prof.begin(side);
        if (dd)
            launch_rqi_dd(hc.nsingle, singles2[level & 1], cur_nodes, blks, dmats, cur_pool, cur_lo,
                          jloc, lo, hi, gapl, gapr, d, e, w, Z, scratch, slots, o.max_rqi,
                          o.fault_mask, dinfo, side);
        else
            launch_rqi(hc.nsingle, singles2[level & 1], cur_nodes, blks, dmats, cur_pool, jloc, lo,
                       hi, gapl, gapr, d, e, w, Z, scratch, (int)slots, nmax, o.max_rqi,
                       o.fault_mask, work, dinfo, team, side);
        prof.end(tq, 4, 1, side);
        cudaEvent_t done = guard.make();
        cudaEventRecord(done, side);
        rqi_done[level & 1] = done;
        return 0;
    };
    // ---- the levels in one graph (mr3_graph.cu), when the options allow it; on a deeper
    // tree or an arena overflow the state after the root bisection is restored and the
    // host-driven loop below does the levels instead
    bool levels_done = false;
    TraceLog trace;
    int graph_levels = 0, graph_runs = 0;
    long long graph_peak = 0;
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap_status);
    // the kernel groups cannot be timed one by one inside a graph: with opts.profile the
    // default keeps the host-driven loop
    const bool graph_auto = nmat >= kGraphMinMatrices && !o.profile;
    if (!dd && !o.abs_split && o.max_depth >= kGraphLevels && cap_status == cudaStreamCaptureStatusNone &&
        (o.graph > 0 || (o.graph == 0 && graph_auto))) {
        GraphLevels G;
        std::memset(&G, 0, sizeof(G));
        G.levels = kGraphLevels;
        G.nblk = nblk;
        G.nmat = nmat;
        G.nmax = nmax;
        G.ncols = ncols;
        G.cap_cl = ncols / 2 + 1;
        // arenas: the worst case (every cluster of two members) when it is at most twice the
        // size of Z (arena 0, which holds the first level's children, the largest set) or
        // Z's size (arenas 1 and 2), else those sizes; a run that overflows reports each
        // arena's need, and the levels are redone once with arenas of those sizes
        long long worst = 0, zsize = 0;
        for (auto &M : mats) {
            worst += (long long)(M.m / 2) * rep_size(M.n);
            zsize += (long long)M.m * M.n;
        }
        for (int k = 0; k < 3; ++k)
            G.pool_cap[k] = std::max<long long>(
                std::min(worst, std::max((k == 0 ? 2 : 1) * zsize, 1ll << 24)), rep_size(nmax));
        G.blks = blks;
        G.mats = dmats;
        G.nodes0 = nodes0;
        G.pool0 = pool0;
        for (int k = 0; k < 3; ++k) G.nodes[k] = ws.get<Node>(G.cap_cl);
        G.singles[0] = singles2[0];
        G.singles[1] = singles2[1];
        G.clusters = clusters;
        G.crep = crep;
        G.cnode = cnode;
        G.jloc = jloc;
        G.next_active = ws.get<int>(ncols);
        G.work = work;
        G.lo = lo;
        G.hi = hi;
        G.gapl = gapl;
        G.gapr = gapr;
        G.tau = ws.get<double>(G.cap_cl);
        G.tri = ws.get<double2>(2 * G.cap_cl);
        G.shift_ws = ws.get<char>(shift_scratch_bytes((int)G.cap_cl, o.max_tries));
        G.ctrs = ws.get<LevelCounters>(kGraphLevels);
        G.slots2 = (int)rqi_slots(ncols, nmax, scratch_cap_bytes, 2);
        G.slots8 = (int)rqi_slots(ncols, nmax, scratch_cap_bytes, 8);
        const size_t sc2 = (size_t)G.slots2 * rqi_scratch_per_index(2) * nmax;
        const size_t sc8 = (size_t)G.slots8 * rqi_scratch_per_index(8) * nmax;
        G.scratch = ws.get<double>(std::max(sc2, sc8));
        G.d = d;
        G.e = e;
        G.w = w;
        G.Z = Z;
        G.dinfo = dinfo;
        G.gaptol = o.gaptol;
        G.rtol = rtol;
        G.max_tries = o.max_tries;
        G.max_rqi = o.max_rqi;
        G.erep = o.erep;
        G.rqi_team = o.rqi_team;
        G.bisect_warps = o.bisect_warps;
        G.tpe = o.tpe;
        G.fault_mask = o.fault_mask;
        // the state after the root bisection, for the fallback
        double *bk_lo = ws.get<double>(ncols), *bk_hi = ws.get<double>(ncols);
        int *bk_cnode = ws.get<int>(ncols), *bk_jloc = ws.get<int>(ncols);
        DevInfo *bk_info = ws.get<DevInfo>(1);
        CKW(ws);
        CK(cudaMemcpyAsync(bk_lo, lo, sizeof(double) * ncols, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bk_hi, hi, sizeof(double) * ncols, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bk_cnode, cnode, sizeof(int) * ncols, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bk_jloc, jloc, sizeof(int) * ncols, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bk_info, dinfo, sizeof(DevInfo), cudaMemcpyDeviceToDevice, s));
        for (int attempt = 0; attempt < 2 && !levels_done; ++attempt) {
            for (int k = 0; k < 3; ++k) G.pool[k] = ws.get<double>(G.pool_cap[k]);
            CKW(ws);
            tk = prof.begin();
            int lv = 0;
            long long need[3] = {0, 0, 0};
            const int grc = run_levels_graph(G, s, side, &lv, need);
            prof.end(tk, 3, 1);
            graph_runs += 1;
            graph_peak = std::max(need[0], std::max(need[1], need[2]));
            if (grc < 0) return -grc;
            for (int k = 0; k < 3; ++k) ws.release(G.pool[k]);
            if (grc == 0) {
                levels_done = true;
                graph_levels = lv;
                break;
            }
            // restore the state after the root bisection
            CK(cudaMemcpyAsync(lo, bk_lo, sizeof(double) * ncols, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(hi, bk_hi, sizeof(double) * ncols, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(cnode, bk_cnode, sizeof(int) * ncols, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(jloc, bk_jloc, sizeof(int) * ncols, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(dinfo, bk_info, sizeof(DevInfo), cudaMemcpyDeviceToDevice, s));
            bool grow = false;
            for (int k = 0; k < 3; ++k) {
                if (need[k] > G.pool_cap[k]) {
                    G.pool_cap[k] = std::min(worst, need[k] + need[k] / 8);
                    grow = true;
                }
            }
            if (!grow) break; // a deeper tree: the host-driven loop takes over
        }
        for (void *p : {(void *)G.nodes[0], (void *)G.nodes[1], (void *)G.nodes[2],
                        (void *)G.next_active,
                        (void *)G.tau, (void *)G.tri,
                        G.shift_ws, (void *)G.ctrs, (void *)G.scratch, (void *)bk_lo,
                        (void *)bk_hi, (void *)bk_cnode, (void *)bk_jloc, (void *)bk_info})
            ws.release(p);
    }
    if (!levels_done)
    for (int level = 0;; ++level) {
        // the singleton buffer of this parity was last read by the RQI two levels back
        if (rqi_done[level & 1]) { cudaStreamWaitEvent(s, rqi_done[level & 1], 0); rqi_done[level & 1] = nullptr; }
        CK(cudaMemsetAsync(ctr, 0, sizeof(LevelCounters), s));
        tk = prof.begin();
        launch_classify(ncur, cur_nodes, blks, lo, hi, o.gaptol, o.abs_split ? 1.0 : 0.0, gapl,
                        gapr, singles2[level & 1],
                        clusters, crep, cnode, ctr, dinfo, s);
        prof.end(tk, 3, 1);
        LevelCounters hc;
        CK(read_back(&hc, ctr, sizeof(hc), s));
        cudaEvent_t level_rqi = nullptr;
        if (hc.nsingle > 0) {
            const int rc = run_singles(level, hc);
            if (rc) return rc;
            level_rqi = rqi_done[level & 1];
        }
        if (hc.ncluster == 0) break;
        const bool at_cap = (level + 1 >= o.max_depth);
        double *next_pool = ws.get<double>(dd ? 2 * (size_t)hc.pool_need : (size_t)hc.pool_need);
        double *next_lo = dd && next_pool ? next_pool + hc.pool_need : nullptr;
        Node *next_nodes = ws.get<Node>(hc.ncluster);
        double *tau = ws.get<double>(hc.ncluster);
        double2 *tri = ws.get<double2>(2 * (size_t)hc.ncluster);
        char *shift_ws = ws.get<char>(shift_scratch_bytes(hc.ncluster, o.max_tries));
        int *next_active = ws.get<int>(hc.nactive);
        CKW(ws);
        TraceLevel *tl = nullptr;
        if (trace_on()) {
            trace.push_back(TraceLevel{level, hc, {}, {}});
            tl = &trace.back();
            for (auto &ev : tl->ev) cudaEventCreate(&ev);
            const int one = 1;
            CK(cudaMemcpyAsync(&dinfo->trace, &one, sizeof(int), cudaMemcpyHostToDevice, s));
            CK(cudaMemsetAsync(&dinfo->tr_max, 0,
                               sizeof(DevInfo) - offsetof(DevInfo, tr_max), s));
            cudaEventRecord(tl->ev[0], s);
        }
        tk = prof.begin();
        launch_refine_ends(hc.ncluster, clusters, cur_nodes, blks, cur_pool, jloc, lo, hi, tri, dinfo, s);
        if (tl) cudaEventRecord(tl->ev[1], s);
        launch_shift(hc.ncluster, clusters, crep, cur_nodes, blks, cur_pool, next_pool,
                     next_nodes, tau, cnode, next_active, jloc, lo, hi, o.max_tries, o.fault_mask,
                     o.erep, tri, shift_ws, dinfo, s);
        if (dd)
            launch_shift_dd(hc.ncluster, clusters, crep, cur_nodes, blks, cur_pool, cur_lo, next_pool,
                            next_lo, next_nodes, tau, dinfo, s);
        prof.end(tk, 5, dd ? 9 : 8); // refine_ends x2, six shift kernels (+ double-double recompute)
        if (tl) cudaEventRecord(tl->ev[2], s);
        tk = prof.begin();
        launch_bisect(hc.nactive, next_active, lanes_for(hc.nactive, o), (int)ncols, cnode,
                      next_nodes, blks, next_pool, jloc, lo, hi, rtol, tau, dinfo, s);
        prof.end(tk, 6, 1);
        if (tl) {
            cudaEventRecord(tl->ev[3], s);
            CK(read_back(&tl->sweeps, dinfo, sizeof(DevInfo), s));
            const int zero = 0;
            CK(cudaMemcpyAsync(&dinfo->trace, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));
        }
        ws.release(next_active);
        ws.release(tri);
        ws.release(shift_ws);
        // return representations no longer read: older levels whose RQI has finished
        for (auto &pnd : pending) {
            if (pnd.done) cudaStreamWaitEvent(s, pnd.done, 0);
            if (pnd.pool != pool0) ws.release(pnd.pool);
            if (pnd.nodes != nodes0) ws.release(pnd.nodes);
        }
        pending.clear();
        pending.push_back({cur_pool, cur_nodes, level_rqi});
        cur_pool = next_pool;
        cur_lo = next_lo;
        cur_nodes = next_nodes;
        ncur = hc.ncluster;
        if (at_cap) {
            // Depth cap: the remaining cluster members are finished as singletons of their
            // current representation (accuracy no longer guaranteed; flagged).
            status = MR3_SDEPTH;
            const int lv = level + 1;
            if (rqi_done[lv & 1]) { cudaStreamWaitEvent(s, rqi_done[lv & 1], 0); rqi_done[lv & 1] = nullptr; }
            CK(cudaMemsetAsync(ctr, 0, sizeof(LevelCounters), s));
            launch_classify(ncur, cur_nodes, blks, lo, hi, -1e308, 0.0, gapl, gapr, singles2[lv & 1],
                            clusters, crep, cnode, ctr, dinfo, s);
            CK(read_back(&hc, ctr, sizeof(hc), s));
            if (hc.nsingle > 0) {
                const int rc = run_singles(lv, hc);
                if (rc) return rc;
            }
            break;
        }
    }
    // the main stream resumes after every singleton launch
    for (auto ev : rqi_done)
        if (ev) cudaStreamWaitEvent(s, ev, 0);
    for (auto &pnd : pending)
        if (pnd.done) cudaStreamWaitEvent(s, pnd.done, 0);
    if (scratch) cudaFreeAsync(scratch, s);
    // ---- output order: sort the eigenpairs of matrices whose eigenvalues came out of order
    int *oflags = ws.get<int>(nmat);
    CKW(ws);
    tk = prof.begin();
    launch_order_flags(nmat, dmats, w, oflags, s);
    prof.end(tk, 7, 1);
    std::vector<int> hflags(nmat);
    CK(read_back(hflags.data(), oflags, sizeof(int) * nmat, s));
    for (int b = 0; b < nmat; ++b) {
        const MatDesc &M = mats[b];
        if (hflags[b] && M.m > 1) {
            double *wtmp = ws.get<double>(M.m);
            double *ztmp = ws.get<double>((size_t)M.m * M.n);
            int *perm = ws.get<int>(M.m);
            CKW(ws);
            tk = prof.begin();
            launch_sort_outputs(b, M.m, dmats, w, Z, wtmp, ztmp, perm, s);
            prof.end(tk, 7, 3);
        }
    }
    DevInfo hi_info;
    CK(read_back(&hi_info, dinfo, sizeof(hi_info), s));
    CK(cudaGetLastError());
    out.dmax = hi_info.dmax;
    out.nclusters = hi_info.nclusters;
    out.largest_cluster = hi_info.largest;
    out.new_rrr = hi_info.new_rrr;
    out.untested_rrr = hi_info.untested;
    out.rqi_iters = (long long)hi_info.rqi_iters;
    out.rqi_iters_max = hi_info.rqi_max;
    out.bisect_fallbacks = hi_info.fallbacks;
    out.sturm_steps = (long long)hi_info.sturm_steps;
    out.shift_steps = (long long)hi_info.shift_steps;
    prof.collect(out);
    for (auto &t : trace) {
        float ms[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < 3; ++k) cudaEventElapsedTime(&ms[k], t.ev[k], t.ev[k + 1]);
        std::fprintf(stderr,
                     "mr3 level %d: singletons %d clusters %d largest %d refine %d pool %lld | "
                     "ends %.3f ms shift %.3f ms bisect %.3f ms\n",
                     t.level, t.hc.nsingle, t.hc.ncluster, t.hc.maxcluster, t.hc.nactive,
                     t.hc.pool_need, ms[0], ms[1], ms[2]);
        static const char *kind[3] = {"bisect", "ends/df", "ends/fp64"};
        for (int k = 0; k < 3; ++k) {
            const DevInfo &v = t.sweeps;
            if (!v.tr_items[k]) continue;
            std::fprintf(stderr, "    %-9s items %llu sweeps mean %.2f max %d lane use %.3f\n",
                         kind[k], v.tr_items[k], (double)v.tr_sweeps[k] / (double)v.tr_items[k],
                         v.tr_max[k],
                         v.tr_warp_lanes[k]
                             ? (double)v.tr_lane_counts[k] / (double)v.tr_warp_lanes[k]
                             : 0.0);
        }
    }
    out.twisted_steps = (long long)hi_info.twisted_steps;
    out.ladder_clusters = hi_info.ladder;
    out.recomputed_rrr = hi_info.recomputed;
    out.graph_levels = graph_levels;
    out.graph_runs = graph_runs;
    out.graph_pool_peak = graph_peak;
    out.envelope_rrr = hi_info.env_accepted;
    for (int k = 0; k < 8; ++k) out.status_counts[k] = hi_info.status[k];
    if (status) out.status_counts[status] += 1;
    if (info) *info = out;
    if (status) return status;
    if (hi_info.status[MR3_SCAP]) return MR3_SCAP;
    if (hi_info.status[MR3_SUNTESTED_RRR]) return MR3_SUNTESTED_RRR;
    return 0;
}

} // namespace
} // namespace mr3

using namespace mr3;

extern "C" {

int mr3_stemr(int n, const double *d, const double *e, int range, double vl, double vu, int il,
              int iu, int *m, double *w, double *Z, int ldz, const mr3_opts *opts,
              mr3_info *info, void *stream) {
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
    *m = 0;
    if (n == 0) {
        if (info) std::memset(info, 0, sizeof(*info));
        return 0;
    }
    const Opts o = resolve(opts);
    std::vector<MatDesc> mats(1);
    std::memset(mats.data(), 0, sizeof(MatDesc));
    mats[0].off = 0;
    mats[0].n = n;
    mats[0].zoff = 0;
    mats[0].ldz = ldz;
    mats[0].woff = 0;
    mats[0].il = il;
    mats[0].iu = iu;
    mats[0].vl = vl;
    mats[0].vu = vu;
    const int rc = solve(1, mats, n, n, d, e, range, w, Z, o, info, (cudaStream_t)stream);
    *m = mats[0].m;
    return rc;
}

int mr3_stemr_host(int n, const double *d, const double *e, int range, double vl, double vu,
                   int il, int iu, int *m, double *w, double *Z, int ldz, const mr3_opts *opts,
                   mr3_info *info, void *stream) {
    if (n < 0) return -1;
    if (n > 0 && !d) return -2;
    if (n > 1 && !e) return -3;
    if (!m) return -9;
    if (n > 0 && !w) return -10;
    if (n > 0 && !Z) return -11;
    if (ldz < std::max(1, n)) return -12;
    *m = 0;
    if (n == 0) return mr3_stemr(0, nullptr, nullptr, range, vl, vu, il, iu, m, nullptr, nullptr, 1, opts, info, stream);
    cudaStream_t s = (cudaStream_t)stream;
    double *dd = nullptr, *de = nullptr, *dw = nullptr, *dz = nullptr;
    int rc = 0;
    if (lib_malloc_async((void **)&dd, sizeof(double) * n, s) != cudaSuccess ||
        lib_malloc_async((void **)&de, sizeof(double) * std::max(1, n - 1), s) != cudaSuccess ||
        lib_malloc_async((void **)&dw, sizeof(double) * n, s) != cudaSuccess ||
        lib_malloc_async((void **)&dz, sizeof(double) * (size_t)n * n, s) != cudaSuccess) {
        cudaGetLastError();
        rc = MR3_EOOM;
    }
    if (!rc) {
        cudaMemcpyAsync(dd, d, sizeof(double) * n, cudaMemcpyHostToDevice, s);
        if (n > 1) cudaMemcpyAsync(de, e, sizeof(double) * (n - 1), cudaMemcpyHostToDevice, s);
        rc = mr3_stemr(n, dd, de, range, vl, vu, il, iu, m, dw, dz, n, opts, info, stream);
        if (rc >= 0 && *m > 0) {
            cudaMemcpyAsync(w, dw, sizeof(double) * (*m), cudaMemcpyDeviceToHost, s);
            cudaMemcpy2DAsync(Z, sizeof(double) * ldz, dz, sizeof(double) * n, sizeof(double) * n,
                              *m, cudaMemcpyDeviceToHost, s);
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); rc = MR3_ECUDA; }
    }
    if (dd) cudaFreeAsync(dd, s);
    if (de) cudaFreeAsync(de, s);
    if (dw) cudaFreeAsync(dw, s);
    if (dz) cudaFreeAsync(dz, s);
    return rc;
}

int mr3_stemr_batched(int nb, const long long *n_off, const double *d, const double *e, int range,
                      const double *vl, const double *vu, const int *il, const int *iu, int *m,
                      double *w, const long long *z_off, double *Z, const mr3_opts *opts,
                      mr3_info *info, void *stream) {
    if (nb < 0) return -1;
    if (nb > 0 && !n_off) return -2;
    if (range < MR3_RANGE_ALL || range > MR3_RANGE_INDEX) return -5;
    if (nb == 0) {
        if (info) std::memset(info, 0, sizeof(*info));
        return 0;
    }
    const long long nrows = n_off[nb] - n_off[0];
    if (n_off[0] != 0) return -2;
    for (int b = 0; b < nb; ++b)
        if (n_off[b + 1] < n_off[b] || n_off[b + 1] - n_off[b] > 0x7fffffffll) return -2;
    if (nrows > 0 && !d) return -3;
    if (nrows > 0 && !e) return -4;
    if (range == MR3_RANGE_VALUE) {
        if (!vl) return -6;
        if (!vu) return -7;
        for (int b = 0; b < nb; ++b) if (!(vl[b] < vu[b])) return -7;
    }
    if (range == MR3_RANGE_INDEX) {
        if (!il) return -8;
        if (!iu) return -9;
        for (int b = 0; b < nb; ++b) {
            const long long nbk = n_off[b + 1] - n_off[b];
            if (nbk == 0) continue;
            if (il[b] < 1 || il[b] > nbk) return -8;
            if (iu[b] < il[b] || iu[b] > nbk) return -9;
        }
    }
    if (!m) return -10;
    if (nrows > 0 && !w) return -11;
    if (!z_off) return -12;
    if (nrows > 0 && !Z) return -13;
    const Opts o = resolve(opts);
    std::vector<MatDesc> mats(nb);
    for (int b = 0; b < nb; ++b) {
        MatDesc &M = mats[b];
        std::memset(&M, 0, sizeof(M));
        M.off = n_off[b];
        M.n = (int)(n_off[b + 1] - n_off[b]);
        M.zoff = z_off[b];
        M.ldz = std::max(1, M.n);
        M.woff = (int)n_off[b];
        M.il = il ? il[b] : 1;
        M.iu = iu ? iu[b] : M.n;
        M.vl = vl ? vl[b] : 0.0;
        M.vu = vu ? vu[b] : 0.0;
    }
    const int rc = solve(nb, mats, nrows, nrows, d, e, range, w, Z, o, info, (cudaStream_t)stream);
    for (int b = 0; b < nb; ++b) m[b] = mats[b].m;
    return rc;
}

int mr3_stemr_batched_host(int nb, const long long *n_off, const double *d, const double *e,
                           int range, const double *vl, const double *vu, const int *il,
                           const int *iu, int *m, double *w, const long long *z_off, double *Z,
                           const mr3_opts *opts, mr3_info *info, void *stream) {
    if (nb < 0) return -1;
    if (nb > 0 && !n_off) return -2;
    if (nb == 0)
        return mr3_stemr_batched(0, n_off, d, e, range, vl, vu, il, iu, m, w, z_off, Z, opts,
                                 info, stream);
    const long long nrows = n_off[nb];
    if (n_off[0] != 0 || nrows < 0) return -2;
    if (nrows > 0 && !d) return -3;
    if (nrows > 0 && !e) return -4;
    if (!m) return -10;
    if (nrows > 0 && !w) return -11;
    if (!z_off) return -12;
    if (nrows > 0 && !Z) return -13;
    long long zlen = 0; // Z elements: the furthest end of any matrix's block
    for (int b = 0; b < nb; ++b) {
        const long long nbk = n_off[b + 1] - n_off[b];
        if (nbk < 0 || z_off[b] < 0) return nbk < 0 ? -2 : -12;
        zlen = std::max(zlen, z_off[b] + nbk * nbk);
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *dd = nullptr, *de = nullptr, *dw = nullptr, *dz = nullptr;
    const size_t rows = (size_t)std::max<long long>(nrows, 1);
    int rc = 0;
    if (lib_malloc_async((void **)&dd, sizeof(double) * rows, s) != cudaSuccess ||
        lib_malloc_async((void **)&de, sizeof(double) * rows, s) != cudaSuccess ||
        lib_malloc_async((void **)&dw, sizeof(double) * rows, s) != cudaSuccess ||
        lib_malloc_async((void **)&dz, sizeof(double) * (size_t)std::max<long long>(zlen, 1), s) !=
            cudaSuccess) {
        cudaGetLastError();
        rc = MR3_EOOM;
    }
    if (!rc && nrows > 0) {
        if (cudaMemcpyAsync(dd, d, sizeof(double) * nrows, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(de, e, sizeof(double) * nrows, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            rc = MR3_ECUDA;
        }
    }
    if (!rc) {
        rc = mr3_stemr_batched(nb, n_off, dd, de, range, vl, vu, il, iu, m, dw, z_off, dz, opts,
                               info, stream);
        if (rc >= 0 && rc != MR3_EOOM && rc != MR3_ECUDA) {
            // eigenvalues of matrix b at w[n_off[b] ..], its m[b] eigenvectors at Z + z_off[b]
            // (leading dimension n_b): one copy per matrix for w and for Z.  rc may hold a
            // positive status (a warning): the results are copied all the same.
            bool copy_failed = false;
            for (int b = 0; b < nb && !copy_failed; ++b) {
                const long long nbk = n_off[b + 1] - n_off[b];
                if (m[b] <= 0) continue;
                if (cudaMemcpyAsync(w + n_off[b], dw + n_off[b], sizeof(double) * m[b],
                                    cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaMemcpyAsync(Z + z_off[b], dz + z_off[b], sizeof(double) * nbk * m[b],
                                    cudaMemcpyDeviceToHost, s) != cudaSuccess) {
                    cudaGetLastError();
                    copy_failed = true;
                }
            }
            if (copy_failed) rc = MR3_ECUDA;
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); rc = MR3_ECUDA; }
    if (dd) cudaFreeAsync(dd, s);
    if (de) cudaFreeAsync(de, s);
    if (dw) cudaFreeAsync(dw, s);
    if (dz) cudaFreeAsync(dz, s);
    return rc;
}

const char *mr3_strerror(int code) {
    if (code < 0) return "invalid argument";
    switch (code) {
    case MR3_SOK: return "success";
    case MR3_SUNTESTED_RRR: return "a cluster representation was accepted without passing the growth test";
    case MR3_SCAP: return "an iteration cap was reached for some eigenpair";
    case MR3_SNONFINITE: return "non-finite input";
    case MR3_SDEPTH: return "representation tree depth cap reached";
    case MR3_EOOM: return "out of device memory";
    case MR3_ECUDA: return "CUDA error";
    case MR3_ENOSCRATCH: return "request exceeds a fixed-size internal buffer";
    default: return "unknown status";
    }
}

const char *mr3_version(void) { return "mr3-gb300 0.1 sm_103a"; }

int mr3_release_memory(void) {
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    int rc = MR3_SOK;
    for (int dev = 0; dev < kMaxDevices; ++dev)
        if (g_pools[dev] && cudaMemPoolTrimTo(g_pools[dev], 0) != cudaSuccess) {
            cudaGetLastError();
            rc = MR3_ECUDA;
        }
    return rc;
}

} // extern "C"
