// mr3_graph.cu -- the levels of the representation tree (Alg. MRRR, breadth first) as one
// CUDA graph: no host read-back between levels.
//
// The host-driven loop (mr3_api.cu) reads each level's counters (singletons, clusters,
// columns to refine, pool size) to size the next launches and allocations.  Here every
// launch is sized for the largest count a level can have and the kernels read the counts
// from the device: classification writes LevelCounters for level L, and the level's
// singleton, shift and refinement launches (and level L+1's classification) take their
// counts from it.  The launch-shape rules (lanes per eigenvalue, per cluster end, RQI team
// size) are the functions the host loop applies to the same counts, so both loops compute
// the same results bit for bit.  The graph unrolls a fixed number of levels; a level with
// nothing to do runs its kernels as empty grids.
//
// Memory.  The representations of level L's children go to arena L % 3 (the roots stay in
// their own pool).  A level's singletons are finished on the side stream while the main
// stream goes on with its clusters: the RQI of level L reads arena (L - 1) % 3, which the
// shift of level L + 2 overwrites, and the singleton list of level L, which classification
// of level L + 2 overwrites; level L + 2 therefore starts after that RQI.  An arena
// holds pool_cap[k] doubles; a level whose representations do not fit flags overflow and
// drops the clusters that do not fit (their columns belong to no node and are left
// alone), and the caller redoes the levels with larger arenas or the host-driven loop, as
// it does when the tree is deeper than the unrolled levels.
#include <algorithm>
#include <vector>
#include "mr3_kernels.h"

namespace mr3 {

int run_levels_graph(const GraphLevels &G, cudaStream_t s_user, cudaStream_t side, int *levels_run,
                     long long need[3]) {
    *levels_run = 0;
    need[0] = need[1] = need[2] = 0;
    const int NLV = G.levels;
    std::vector<cudaEvent_t> ev_cls(NLV, nullptr), ev_rqi(NLV, nullptr);
    cudaEvent_t ev_fork = nullptr;
    // the caller's stream may be the legacy default stream, which cannot be captured: the
    // graph is captured on a stream of its own and launched on the caller's
    cudaStream_t s = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = 0;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : ev_cls)
            if (e) cudaEventDestroy(e);
        for (auto e : ev_rqi)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (s) cudaStreamDestroy(s);
    };
    auto fail = [&](cudaError_t e) {
        cudaGetLastError();
        cleanup();
        return e == cudaErrorMemoryAllocation ? -MR3_EOOM : -MR3_ECUDA;
    };
    cudaError_t err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    for (int L = 0; L < NLV && err == cudaSuccess; ++L) {
        err = cudaEventCreateWithFlags(&ev_cls[L], cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev_rqi[L], cudaEventDisableTiming);
    }
    if (err != cudaSuccess) return fail(err);
    err = cudaMemsetAsync(G.ctrs, 0, sizeof(LevelCounters) * NLV, s_user);
    if (err != cudaSuccess) return fail(err);

    err = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return fail(err);
    // the side stream joins the capture through an event recorded on s
    cudaEventRecord(ev_fork, s);
    cudaStreamWaitEvent(side, ev_fork, 0);
    for (int L = 0; L < NLV; ++L) {
        const Node *cur_nodes = L == 0 ? G.nodes0 : G.nodes[(L - 1) % 3];
        const double *cur_pool = L == 0 ? G.pool0 : G.pool[(L - 1) % 3];
        Node *next_nodes = G.nodes[L % 3];
        double *next_pool = G.pool[L % 3];
        LevelCounters *ctr = G.ctrs + L;
        const int *dncur = L == 0 ? nullptr : &G.ctrs[L - 1].ncluster;
        const int ncur_cap = L == 0 ? G.nblk : (int)G.cap_cl;
        // the singleton list and the arena of level L - 2 are still read by its RQI
        if (L >= 2) cudaStreamWaitEvent(s, ev_rqi[L - 2], 0);
        launch_classify(ncur_cap, cur_nodes, G.blks, G.lo, G.hi, G.gaptol, 0.0, G.gapl, G.gapr,
                        G.singles[L & 1], G.clusters, G.crep, G.cnode, ctr, G.dinfo, s, dncur,
                        G.pool_cap[L % 3]);
        cudaEventRecord(ev_cls[L], s);
        // ---- singletons on the side stream
        cudaStreamWaitEvent(side, ev_cls[L], 0);
        launch_rqi_dev((int)G.ncols, &ctr->nsingle, G.nmat, G.rqi_team, G.singles[L & 1], cur_nodes,
                       G.blks, G.mats, cur_pool, G.jloc, G.lo, G.hi, G.gapl, G.gapr, G.d, G.e,
                       G.w, G.Z, G.scratch, G.slots2, G.slots8, G.nmax, G.max_rqi, G.fault_mask,
                       G.work, G.dinfo, side);
        cudaEventRecord(ev_rqi[L], side);
        // ---- clusters on the main stream
        launch_refine_ends((int)G.cap_cl, G.clusters, cur_nodes, G.blks, cur_pool, G.jloc, G.lo,
                           G.hi, G.tri, G.dinfo, s, &ctr->ncluster);
        launch_shift((int)G.cap_cl, G.clusters, G.crep, cur_nodes, G.blks, cur_pool, next_pool,
                     next_nodes, G.tau, G.cnode, G.next_active, G.jloc, G.lo, G.hi, G.max_tries,
                     G.fault_mask, G.erep, G.tri, G.shift_ws, G.dinfo, s, &ctr->ncluster);
        launch_bisect((int)G.ncols, G.next_active, 1, (int)G.ncols, G.cnode, next_nodes, G.blks,
                      next_pool, G.jloc, G.lo, G.hi, G.rtol, G.tau, G.dinfo, s, &ctr->nactive,
                      G.bisect_warps, G.tpe);
    }
    // the main stream resumes after the last singleton launch
    cudaStreamWaitEvent(s, ev_rqi[NLV - 1], 0);
    err = cudaStreamEndCapture(s, &graph);
    if (err != cudaSuccess) return fail(err);
    err = cudaGraphInstantiate(&exec, graph, 0);
    if (err != cudaSuccess) return fail(err);
    err = cudaGraphLaunch(exec, s_user);
    if (err != cudaSuccess) return fail(err);
    std::vector<LevelCounters> h(NLV);
    err = read_back(h.data(), G.ctrs, sizeof(LevelCounters) * NLV, s_user);
    if (err != cudaSuccess) return fail(err);
    bool overflow = false;
    int used = 0;
    for (int L = 0; L < NLV; ++L) {
        // the first level that overflowed still counted its whole need; later ones may not
        // have seen correct data
        if (!overflow) need[L % 3] = std::max(need[L % 3], h[L].pool_need);
        overflow |= h[L].overflow != 0;
        if (L == 0 || h[L - 1].ncluster > 0) used = L + 1;
    }
    *levels_run = used;
    rc = (overflow || h[NLV - 1].ncluster > 0) ? 1 : 0;
    cleanup();
    return rc;
}

} // namespace mr3
