// mr3_kernels.h -- host-side launchers of the MRRR kernels (one per .cu stage).
#pragma once
#include <cuda_runtime.h>
#include "mr3.h"
#include "mr3_internal.cuh"

namespace mr3 {

// ---- prologue (mr3_prologue.cu)
// Per matrix: Gershgorin norm of the whole matrix; flags rows that start a block.
void launch_mat_norm(int nmat, MatDesc *mats, const double *d, const double *e, int *bad_input,
                     cudaStream_t s);
void launch_split_flags(int nmat, const MatDesc *mats, long long nrows, const double *d,
                        const double *e, int *flags, cudaStream_t s);
// Exclusive scan of n ints (in place allowed); *total (device) gets the sum.
void launch_exclusive_scan(const int *in, int *out, long long n, int *total, int *tmp,
                           cudaStream_t s);
size_t scan_tmp_ints(long long n);
// Build block descriptors from the scanned flags.
void build_blocks(long long nrows, const int *flags, const int *scanned, const int *nblk_dev,
                  int nblk_host, int nmat, MatDesc *mats, BlkDesc *blks, cudaStream_t s);
// Per block: Gershgorin, selected local index range, output columns (range != ALL
// needs the per-matrix index/value data in mats).
void launch_blk_setup(int nblk, BlkDesc *blks, int nmat, MatDesc *mats, const double *d,
                      const double *e, int range, cudaStream_t s);
// Range INDEX on matrices that split into several blocks: per-block index ranges.
void launch_index_multi(int nmat, MatDesc *mats, BlkDesc *blks, const double *d,
                        const double *e, cudaStream_t s);
// Per matrix: columns of each block and m.
void launch_assign_columns(int nmat, MatDesc *mats, BlkDesc *blks, int range, cudaStream_t s);
// Root representation of every block (Alg. MRRR, root representation and its perturbation).
void launch_root(int nblk, BlkDesc *blks, const double *d, const double *e, double *pool0,
                 float *f32scratch, unsigned long long seed, cudaStream_t s);
// Level-0 nodes, per-column state and starting intervals.
void launch_init_columns(int nblk, const BlkDesc *blks, Node *nodes, int *cnode, int *jloc,
                         double *lo, double *hi, int mtotal, cudaStream_t s);
// Gaps to the eigenvalues just outside a subset (range != ALL).
void launch_outer_gaps(int nblk, const BlkDesc *blks, Node *nodes, const double *pool0,
                       double rtol, DevInfo *info, cudaStream_t s);
void launch_zero_z(int nmat, const MatDesc *mats, double *Z, cudaStream_t s);

// ---- representation tree (mr3_levels.cu)
// Multisection with L lanes (1, 2, 4, ..., 32) per eigenvalue over ngroups columns
// (list[g], or g itself when list is NULL).
void launch_bisect(int ngroups, const int *list, int L, int mtotal, const int *cnode,
                   const Node *nodes, const BlkDesc *blks, const double *pool, const int *jloc,
                   double *lo, double *hi, double rtol, const double *tau_of_node, DevInfo *info,
                   cudaStream_t s, const int *dngroups = nullptr, int warps_per_sm = 0,
                   int tpe = 0);
// Shared grid of Sturm counts giving the starting intervals of the root level.
void launch_grid(int nblk, const BlkDesc *blks, const Node *nodes, const double *pool, int *grid,
                 double *lo, double *hi, int max_m, DevInfo *info, cudaStream_t s);
// absfac > 0: at the root (depth 0) also separate j, j+1 when their absolute gap is at least
// absfac times the block's average gap spdiam / (n_b - 1) (the amendment of the relative
// criterion by absolute gaps, Sec. 3.2.3 and Sec. 4.2.1); the pieces this extra split cuts
// out of a relative cluster stay clusters, however small.
void launch_classify(int nnode, const Node *nodes, const BlkDesc *blks, const double *lo,
                     const double *hi, double gaptol, double absfac, double *gapl, double *gapr,
                     SingleItem *singles, ClusterItem *clusters, long long *cluster_rep,
                     int *cnode, LevelCounters *ctr, DevInfo *info, cudaStream_t s,
                     const int *dnnode = nullptr, long long pool_cap = 0);
// Refine the two extreme eigenvalues of every cluster (Alg. "Shifting the spectrum", first step).
// carry: 2 ncluster double2 of scratch.
void launch_refine_ends(int ncluster, const ClusterItem *clusters, const Node *nodes,
                        const BlkDesc *blks, const double *pool, const int *jloc, double *lo,
                        double *hi, double2 *carry, DevInfo *info, cudaStream_t s,
                        const int *dncluster = nullptr);
// tri: scratch of 2 ncluster double2 (existence and growth of the first two candidates);
// ws: shift_scratch_bytes(ncluster, max_tries) bytes (decisions, back-off results, queues).
void launch_shift(int ncluster, const ClusterItem *clusters, const long long *cluster_rep,
                  const Node *nodes, const BlkDesc *blks, const double *pool, double *childpool,
                  Node *child_nodes, double *child_tau, int *cnode, int *active_list,
                  const int *jloc, double *lo, double *hi, int max_tries, unsigned fault_mask,
                  int erep, double2 *tri, void *ws, DevInfo *info, cudaStream_t s,
                  const int *dncluster = nullptr);
// Stream-ordered allocation from the library's memory pool of the current device (one
// pool per device whose release threshold keeps freed memory for later calls); free with
// cudaFreeAsync.
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s);

// Bytes of the ws scratch launch_shift needs for ncluster clusters.
size_t shift_scratch_bytes(int ncluster, int max_tries);
// Ascending eigenvalues: running-maximum fix for single-block matrices, flags for the rest.
void launch_order_flags(int nmat, const MatDesc *mats, double *w, int *flags, cudaStream_t s);
// Sort the m eigenpairs of matrix mi (temporaries: m values, n x m entries, m ints).
void launch_sort_outputs(int mi, int m, const MatDesc *mats, double *w, double *Z, double *wtmp,
                         double *ztmp, int *perm, cudaStream_t s);

// ---- singletons (mr3_rqi.cu)
void launch_rqi(int nsingle, const SingleItem *singles, const Node *nodes, const BlkDesc *blks,
                const MatDesc *mats, const double *pool, const int *jloc, const double *lo,
                const double *hi, const double *gapl, const double *gapr, const double *d,
                const double *e, double *w, double *Z, double *scratch, int nslots, int nmax,
                int max_rqi, unsigned fault_mask, int *work_counter, DevInfo *info,
                int team, cudaStream_t s);
// The same with the singleton count on the device (at most max_single): both team sizes are
// launched (grids of at most nslots2 / nslots8 warp slots over the same scratch), and the
// team the count selects (rqi_team_rule) does the work.
void launch_rqi_dev(int max_single, const int *dnsingle, int nmat, int forced_team,
                    const SingleItem *singles, const Node *nodes, const BlkDesc *blks,
                    const MatDesc *mats, const double *pool, const int *jloc, const double *lo,
                    const double *hi, const double *gapl, const double *gapr, const double *d,
                    const double *e, double *w, double *Z, double *scratch, int nslots2,
                    int nslots8, int nmax, int max_rqi, unsigned fault_mask, int *work_counter,
                    DevInfo *info, cudaStream_t s);

// Team size (lanes per singleton, 2 or 8) for a launch of nsingle singletons of a solve over
// nmat matrices; scratch doubles
// per index per warp slot, and singletons a warp slot holds at a time, for that team size.
int rqi_team(long long nsingle, int nmat);
int rqi_scratch_per_index(int team);
int rqi_singles_per_slot(int team);

// Forces the kernels of one translation unit to be loaded on the current device (the
// runtime otherwise loads each kernel at its first launch, which can allocate device
// memory); returns the first error.  Used by the set-up of mr3_stemr_static.
template <class... K> cudaError_t load_kernels(K... k) {
    cudaError_t err = cudaSuccess;
    cudaFuncAttributes a;
    const void *fns[] = {(const void *)k...};
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    }
    return err;
}
// Copies bytes from device memory to host memory in stream order and waits for them
// (mr3_api.cu: through a mapped pinned buffer, no copy engine).
cudaError_t read_back(void *dst, const void *src, size_t bytes, cudaStream_t s);
// C (M x N, FP32, column-major, ldc) = sum_{k0 <= k < k1} A[m, k] B[k, j] on the tensor
// cores (mr3_tc_gemm.cu): bf16 operands, both K-major (A row m at A + m lda, B column j at
// B + j ldb, K extent K), lda and ldb multiples of 64, k0 a multiple of 64, 16-byte aligned
// bases; products exact while every chunk sum is an integer below 2^24.  Returns 0, or -1
// when the arguments or the launch are rejected; *err (device) is set to 1 when a wait in
// the kernel gave up.
int tc_gemm_bf16(int M, int N, int K, int k0, int k1, const unsigned short *A, int lda,
                 const unsigned short *B, int ldb, float *C, int ldc, int *err, cudaStream_t s);
cudaError_t preload_tc_gemm();
// Eigenvector part of the backward pass one eigenpair at a time (mr3_adjoint.cu): column c
// of Y (n x k, ld n) such that Y Z^T is the eigenvector part of Tbar; scratch of
// adjoint_scratch_doubles(n, k) doubles.
size_t adjoint_scratch_doubles(int n, int k);
void launch_adjoint(int n, int k, const double *d, const double *e, const double *w,
                    const double *Z, int ldz, const double *G, int ldg, double tnorm,
                    double *scratch, double *Y, cudaStream_t s);
cudaError_t preload_prologue();
cudaError_t preload_levels();
cudaError_t preload_rqi();

// ---- double-double representation tree (mr3_ddpath.cu, opts->prec = MR3_DD).  A pool
// holding representations keeps the leading words in the binary64 layout and the low
// words in a second plane at the same offsets (pool_lo).
void launch_root_dd(int nblk, BlkDesc *blks, const double *d, const double *e, double *pool0,
                    double *pool0_lo, unsigned long long seed, cudaStream_t s);
void launch_shift_dd(int ncluster, const ClusterItem *clusters, const long long *cluster_rep,
                     const Node *nodes, const BlkDesc *blks, const double *pool,
                     const double *pool_lo, double *childpool, double *childpool_lo,
                     Node *child_nodes, const double *child_tau, DevInfo *info, cudaStream_t s);
// Threads for a singleton launch within a scratch budget (4 nmax doubles per thread).
long long rqi_dd_threads(long long nsingle, int nmax, long long cap_bytes);
void launch_rqi_dd(int nsingle, const SingleItem *singles, const Node *nodes, const BlkDesc *blks,
                   const MatDesc *mats, const double *pool, const double *pool_lo, const int *jloc,
                   const double *lo, const double *hi, const double *gapl, const double *gapr,
                   const double *d, const double *e, double *w, double *Z, double *scratch,
                   long long nthreads, int max_rqi, unsigned fault_mask, DevInfo *info,
                   cudaStream_t s);

// ---- the level loop captured in one CUDA graph (mr3_graph.cu).  Every buffer is sized
// for the largest counts a level can have (clusters <= ncols / 2 + 1), the kernels read
// the level's counts from the device, and the launch shapes follow the same rules as the
// host-driven loop, so the results are the same bit for bit.
struct GraphLevels {
    int levels;                // levels unrolled in the graph
    int nblk, nmat, nmax;
    long long ncols, cap_cl;   // columns; clusters per level at most
    long long pool_cap[3];     // doubles per representation arena
    const BlkDesc *blks;
    const MatDesc *mats;
    Node *nodes0;              // level 0: the roots
    double *pool0;
    Node *nodes[3];            // children of level L go to arena L % 3
    double *pool[3];
    SingleItem *singles[2];    // singleton list of level L: singles[L & 1]
    ClusterItem *clusters;
    long long *crep;
    int *cnode, *jloc, *next_active, *work;
    double *lo, *hi, *gapl, *gapr, *tau;
    double2 *tri;
    void *shift_ws;            // shift_scratch_bytes(cap_cl, max_tries)
    LevelCounters *ctrs;       // one per level
    double *scratch;           // RQI scratch for slots2 team-2 / slots8 team-8 warp slots
    int slots2, slots8;
    const double *d, *e;
    double *w, *Z;
    DevInfo *dinfo;
    double gaptol, rtol;
    int max_tries, max_rqi, erep, rqi_team, bisect_warps, tpe;
    unsigned fault_mask;
};
// Captures G.levels levels on stream s (singletons on side) into one graph, launches it
// and waits.  Returns 0 when the tree ended within those levels, 1 when the levels must
// be redone (a deeper tree, or representations that overflowed an arena), or a negative
// CUDA error.  *levels_run: levels that classified at least one node; need[k]: the
// largest need of arena k seen up to and including the first level that overflowed.
int run_levels_graph(const GraphLevels &G, cudaStream_t s, cudaStream_t side, int *levels_run,
                     long long need[3]);

} // namespace mr3
