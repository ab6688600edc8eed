// mr3_levels.cu -- traversal of the representation tree, one level per launch group
// (Alg. MRRR, breadth first): bisection to classification accuracy (Alg. Bisection),
// classification by relative gaps (Sec. 3.2.3), and for every cluster a new
// representation by a shift of the spectrum (Alg. "Shifting the spectrum", C-task).
#include <float.h>
#include <algorithm>
#include "mr3_kernels.h"
#include "mr3_df.cuh"

namespace mr3 {

#define FULL_MASK 0xffffffffu

// Offset of the shifts from the cluster's end eigenvalues, in units of eps |lambda|
// (Alg. "Shifting the spectrum" suggests 100).
// Lanes given to the cluster-end refinement: MR3_REFINE_WARPS_PER_SM and
// MR3_REFINE1_LANES_PER_SM (mr3_internal.cuh, refine_lanes).

// Relative width at which the double-float phase of the cluster-end refinement stops.
#ifndef MR3_REFINE_DF_RTOL
#define MR3_REFINE_DF_RTOL 1e-13
#endif
constexpr double kRefineDfRtol = MR3_REFINE_DF_RTOL;

#ifndef MR3_TAU_OFFSET
#define MR3_TAU_OFFSET 100.0
#endif

// ------------------------------------------------------------------ bisection

// Whether a count of node N at x runs in double-float.
__device__ __forceinline__ bool node_df(const Node &N, double x) {
    return N.dfok && df_shift_ok(scalbn(x, N.dfexp));
}

// Sturm count at x for one node: double-float on the node's scaled copy when that is
// usable (Ch. 5 x-bit eigenvalue approximation), else binary64.
__device__ __forceinline__ int node_count(const Node &N, int n, const double *__restrict__ rep,
                                          double x) {
    if (node_df(N, x)) {
        const int k = negcount_df(n, (const float4 *)(rep + rep_df_offset(n)),
                                  df_from(scalbn(x, N.dfexp)));
        if (k >= 0) return k;
    }
    return negcount_ldl(n, rep, rep + 2 * n, x);
}

// Multisection (Alg. Bisection generalised to L interior points per sweep): a group of L
// lanes owns one eigenvalue j of a node; each sweep the lanes count at the L interior
// points of [lo, hi] (L + 1 equal parts) and a ballot of "count < j" picks the part that
// holds lambda_j, so a sweep gains log2(L + 1) bits.  Stop when
// hi - lo <= max(rtol max(|lo|, |hi|), atol).
//
// Refinement on a child (tau_of_node != NULL): the parent interval is mapped to the child
// by subtracting tau and widened by 8 eps (|bound| + |tau|); the two ends are verified by
// Sturm counts on the child; if they do not bracket lambda_j the interval is widened by the
// paper's factor nu = 10 k_rr n eps, k_rr = 10 ((lambda (1 -+ nu) - tau)(1 -+ nu), end of
// Sec. 3.2.3), then by powers of 2^8.
//
// Counts in double-float (on the node's copy scaled by 2^dfexp, where every binary32
// product stays normal) are exact for a relative perturbation of the representation of a
// few units of 2^-47, so the final interval is widened by 32 n 2^-47 relative.
__global__ void k_bisect2(int ngroups, const int *__restrict__ list, int L_host, int mtotal,
                          const int *__restrict__ cnode, const Node *__restrict__ nodes,
                          const BlkDesc *__restrict__ blks, const double *__restrict__ pool,
                          const int *__restrict__ jloc, double *lo, double *hi, double rtol,
                          const double *__restrict__ tau_of_node, DevInfo *info,
                          const int *dngroups, int warps_per_sm, int tpe) {
    // with a device count the lanes per eigenvalue follow the host's rule
    if (dngroups) ngroups = *dngroups;
    const int L = dngroups ? bisect_lanes(ngroups, warps_per_sm, tpe) : L_host;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int gid = tid / L;
    const int k = lane % L;
    const int gbase = lane - k;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << gbase);
    bool active = gid < ngroups;
    int c = 0;
    if (active) {
        c = list ? list[gid] : gid;
        active = c < mtotal && cnode[c] >= 0;
    }
    Node N;
    int n = 1, j = 1;
    const double *rep = pool;
    double l = 0.0, h = 0.0;
    unsigned long long steps = 0;
    if (active) {
        N = nodes[cnode[c]];
        n = blks[N.blk].n;
        rep = pool + N.rep;
        j = jloc[c];
        l = lo[c];
        h = hi[c];
    } else {
        N.dfok = 0;
    }
    if (tau_of_node) {
        // ---- map the parent interval to the child and verify it brackets lambda_j
        double tau = 0.0, pl = l, ph = h;
        if (active) {
            tau = tau_of_node[cnode[c]];
            const double m0 = 8.0 * kEps * (fmax(fabs(pl), fabs(ph)) + fabs(tau));
            l = (pl - tau) - m0;
            h = (ph - tau) + m0;
        }
        for (int attempt = 0; attempt < 8; ++attempt) {
            int okL = 1, okH = 1;
            if (active) {
                if (L >= 2) {
                    int cnt = 0;
                    if (k < 2) { cnt = node_count(N, n, rep, k == 0 ? l : h); steps += n; }
                    const int c0 = __shfl_sync(gmask, cnt, gbase), c1 = __shfl_sync(gmask, cnt, gbase + 1);
                    okL = c0 < j;
                    okH = c1 >= j;
                } else {
                    okL = node_count(N, n, rep, l) < j;
                    okH = node_count(N, n, rep, h) >= j;
                    steps += 2ull * n;
                }
            } else if (L >= 2) {
                (void)__shfl_sync(gmask, 0, gbase);
                (void)__shfl_sync(gmask, 0, gbase + 1);
            }
            const bool ok = okL && okH;
            if (__all_sync(0xffffffffu, ok || !active)) break;
            if (active && !ok) {
                if (attempt == 0) {
                    const double nu = 100.0 * n * kEps;
                    double a = pl - nu * fabs(pl) - tau;
                    a -= nu * fabs(a);
                    double b = ph + nu * fabs(ph) - tau;
                    b += nu * fabs(b);
                    if (!okL) l = fmin(l, a);
                    if (!okH) h = fmax(h, b);
                } else {
                    const double g = ldexp(fmax(h - l, 4.0 * kSafmin), 8);
                    if (!okL) l -= g;
                    if (!okH) h += g;
                }
            }
        }
    }
    // ---- multisection.  Double-float counts while the interval is wider than their
    // accuracy (64 n 2^-47 relative); below that the interval is widened by the
    // double-float error bound and the bisection goes on in binary64.
    const double atol = 4.0 * kSafmin;
    const double kap = 32.0 * n * 0x1p-47;
    bool used_df = false;
    bool df_phase = N.dfok != 0;
    int sw = 0, rounds = 0;
    for (int sweep = 0; sweep < 400; ++sweep) {
        if (active && df_phase && h - l <= 2.0 * kap * fmax(fabs(l), fabs(h))) {
            if (used_df) {
                l -= kap * fabs(l);
                h += kap * fabs(h);
            }
            df_phase = false;
            used_df = false;
        }
        const double w = h - l;
        bool done = !active || !(w > fmax(rtol * fmax(fabs(l), fabs(h)), atol));
        const double x = l + (k + 1) * (w / (L + 1));
        // no representable interior point left: the group stops
        if (__ballot_sync(0xffffffffu, !(x > l && x < h)) & gmask) done = true;
        if (__all_sync(0xffffffffu, done)) break;
        int cnt = 0;
        if (!done) {
            if (df_phase) {
                used_df |= node_df(N, x);
                cnt = node_count(N, n, rep, x);
            } else {
                cnt = negcount_ldl(n, rep, rep + 2 * n, x);
            }
            steps += n;
            ++sw;
        }
        ++rounds;
        const unsigned bal = __ballot_sync(0xffffffffu, cnt < j);
        const int t = __popc(bal & gmask);
        const double xl = __shfl_sync(0xffffffffu, x, gbase + (t > 0 ? t - 1 : 0));
        const double xh = __shfl_sync(0xffffffffu, x, gbase + (t < L ? t : L - 1));
        if (!done) {
            if (t > 0) l = xl;
            if (t < L) h = xh;
        }
    }
    if (info->trace) trace_sweeps(info, 0, active && k == 0, sw, rounds);
    const bool grp_df = (__ballot_sync(0xffffffffu, used_df) & gmask) != 0;
    if (active && k == 0) {
        if (grp_df) {
            l -= kap * fabs(l);
            h += kap * fabs(h);
        }
        lo[c] = l;
        hi[c] = h;
    }
    for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, o);
    if (lane == 0 && steps) atomicAdd(&info->sturm_steps, steps);
}

void launch_bisect(int ngroups, const int *list, int L, int mtotal, const int *cnode,
                   const Node *nodes, const BlkDesc *blks, const double *pool, const int *jloc,
                   double *lo, double *hi, double rtol, const double *tau_of_node, DevInfo *info,
                   cudaStream_t s, const int *dngroups, int warps_per_sm, int tpe) {
    if (ngroups <= 0) return;
    // with a device count (at most ngroups): enough threads for any count's lanes
    long long threads = (long long)ngroups * L;
    if (dngroups)
        threads = tpe > 0 ? (long long)ngroups * bisect_lanes(0, warps_per_sm, tpe)
                          : std::max<long long>(152ll * 32 * warps_per_sm, ngroups);
    // small launches in single-warp blocks, so that they spread over all SMs
    const int bs = threads >= 152ll * 128 * 2 ? 128 : 32;
    k_bisect2<<<(unsigned)((threads + bs - 1) / bs), bs, 0, s>>>(ngroups, list, L, mtotal, cnode,
                                                                 nodes, blks, pool, jloc, lo, hi,
                                                                 rtol, tau_of_node, info, dngroups,
                                                                 warps_per_sm, tpe);
}

// Root level, most of a block's spectrum requested: G + 1 equally spaced points over the
// block's shifted Gershgorin interval are counted once (one thread each) and every
// requested eigenvalue takes the grid cell that holds it as its starting interval, so the
// first log2(G) bits are shared by all eigenvalues instead of bisected one by one.
__global__ void k_grid_counts(int nblk, const BlkDesc *__restrict__ blks, const Node *__restrict__ nodes,
                              const double *__restrict__ pool, int *grid, DevInfo *info) {
    const int b = blockIdx.y;
    const BlkDesc B = blks[b];
    const int m = B.j1 >= B.j0 ? B.j1 - B.j0 + 1 : 0;
    const bool use = m > 0 && 4 * m >= B.n;
    const int G = ((max(m, 32) + 31) / 32) * 32;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long steps = 0;
    if (use && p <= G) {
        int *cnt = grid + B.col0 + 64 * b;
        if (p == 0) {
            cnt[0] = 0;
        } else if (p == G) {
            cnt[G] = B.n;
        } else {
            const Node N = nodes[b];
            const double a = B.gl - B.mu, z = B.gu - B.mu;
            const double pad = 64.0 * (B.n + 1) * kEps * fmax(fabs(a), fabs(z)) + 4.0 * kSafmin;
            const double ga = a - pad, gz = z + pad;
            const double x = ga + (gz - ga) * ((double)p / G);
            cnt[p] = node_count(N, B.n, pool + N.rep, x);
            steps = B.n;
        }
    }
    for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, o);
    if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&info->sturm_steps, steps);
}

__global__ void k_grid_bracket(int nblk, const BlkDesc *__restrict__ blks, const int *__restrict__ grid,
                               double *lo, double *hi) {
    const int b = blockIdx.y;
    if (b >= nblk) return;
    const BlkDesc B = blks[b];
    const int m = B.j1 >= B.j0 ? B.j1 - B.j0 + 1 : 0;
    if (m == 0 || 4 * m < B.n) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int G = ((max(m, 32) + 31) / 32) * 32;
    const int *cnt = grid + B.col0 + 64 * b;
    const int j = B.j0 + t;
    // largest p with cnt[p] < j (cnt[0] = 0 < j, cnt[G] = n >= j)
    int a = 0, z = G;
    while (z - a > 1) {
        const int mid = (a + z) >> 1;
        if (cnt[mid] < j) a = mid; else z = mid;
    }
    const double ga0 = B.gl - B.mu, gz0 = B.gu - B.mu;
    const double pad = 64.0 * (B.n + 1) * kEps * fmax(fabs(ga0), fabs(gz0)) + 4.0 * kSafmin;
    const double ga = ga0 - pad, gz = gz0 + pad;
    const int c = B.col0 + t;
    lo[c] = (a == 0) ? ga : ga + (gz - ga) * ((double)a / G);
    hi[c] = (z == G) ? gz : ga + (gz - ga) * ((double)z / G);
}

void launch_grid(int nblk, const BlkDesc *blks, const Node *nodes, const double *pool, int *grid,
                 double *lo, double *hi, int max_m, DevInfo *info, cudaStream_t s) {
    if (nblk <= 0 || max_m <= 0) return;
    const int G = ((std::max(max_m, 32) + 31) / 32) * 32;
    dim3 g1((G + 1 + 63) / 64, nblk);
    k_grid_counts<<<g1, 64, 0, s>>>(nblk, blks, nodes, pool, grid, info);
    dim3 g2((max_m + 127) / 128, nblk);
    k_grid_bracket<<<g2, 128, 0, s>>>(nblk, blks, grid, lo, hi);
}

// ------------------------------------------------------------------ classification

// One warp per node.  Consecutive eigenvalues j, j+1 of the node are separated when
//   reldist(j, j+1) = (lo_{j+1} - hi_j) / max(|lo_j|, |hi_j|, |lo_{j+1}|, |hi_{j+1}|) >= gaptol
// (Sec. 3.2.3, Classification); gaptol == kGaptolAuto selects auto_gaptol(n_b) for the
// node's block.  With absfac > 0, a root node also separates j, j+1 when
//   mid_{j+1} - mid_j >= absfac * spdiam / (n_b - 1),   mid = (lo + hi) / 2,
// i.e. when their absolute gap reaches absfac times the average gap of the block (the
// absolute-gap amendment, Sec. 3.2.3 and Sec. 4.2.1).  The gap is taken between the
// midpoints: at classification accuracy the intervals' widths (rtol |lambda|) are a
// sizeable part of the average gap once n_b is in the thousands, and the bound gap
// lo_{j+1} - hi_j would split less the larger the matrix.  A piece that such a split cuts out
// of a relative cluster is a cluster even when it has one member: its relative gap in the
// root representation is below gaptol, so its vector needs a representation shifted close
// to it.  The boundary flags of 32 columns at a time are combined with a ballot; groups
// of one column bounded by relative gaps on both sides become singletons, the other groups
// clusters.  Items are appended with one atomic per warp and kind.  gapl/gapr receive the
// absolute gaps of every column to its neighbours (used by the RQI acceptance test).
__device__ __forceinline__ void k_classify_item(int w, int nnode, const Node *__restrict__ nodes,
                           const BlkDesc *__restrict__ blks, const double *__restrict__ lo, const double *__restrict__ hi,
                           double gaptol, double absfac, double *gapl, double *gapr,
                           SingleItem *singles,
                           ClusterItem *clusters, long long *cluster_rep, int *cnode,
                           LevelCounters *ctr, DevInfo *info, const int *dnnode,
                           long long pool_cap) {
    const int lane = threadIdx.x & 31;
    const Node N = nodes[w];
    if (N.c1 < N.c0) return;
    const int nb = blks[N.blk].n;
    const double gt = (gaptol == kGaptolAuto) ? auto_gaptol(nb) : gaptol;
    const double absgap = (absfac > 0.0 && N.depth == 0 && nb > 1)
                              ? absfac * blks[N.blk].spdiam / (double)(nb - 1) : INFINITY;
    int gstart = N.c0;
    bool gstart_rel = true; // the boundary before gstart is a relative one (or the node's start)
    int maxsize = 0, nclus = 0;
    for (int base = N.c0; base <= N.c1; base += 32) {
        const int c = base + lane;
        const bool valid = c <= N.c1;
        double l = 0.0, h = 0.0, ln = 0.0, hn = 0.0;
        bool end = false, end_rel = false;
        if (valid) {
            l = lo[c];
            h = hi[c];
            if (c < N.c1) {
                ln = lo[c + 1];
                hn = hi[c + 1];
                const double den = fmax(fmax(fabs(l), fabs(h)), fmax(fabs(ln), fabs(hn)));
                const double rd = (ln - h) / den;
                end_rel = !(rd < gt); // also separates on NaN (never join on bad data)
                end = end_rel || (0.5 * (ln + hn) - 0.5 * (l + h) >= absgap);
            } else {
                end = end_rel = true;
            }
            const double left = (c > N.c0) ? hi[c - 1] : N.lnb;
            const double right = (c < N.c1) ? ln : N.rnb;
            gapl[c] = l - left;
            gapr[c] = right - h;
            cnode[c] = -1;
        }
        const unsigned mask = __ballot_sync(FULL_MASK, end);
        const unsigned mrel = __ballot_sync(FULL_MASK, end_rel);
        int gs = gstart;
        bool lrel = gstart_rel;
        if (end) {
            const unsigned prev = mask & ((1u << lane) - 1u);
            if (prev) {
                const int b = 31 - __clz(prev);
                gs = base + b + 1;
                lrel = (mrel >> b) & 1u;
            }
        }
        const int size = end ? c - gs + 1 : 0;
        const bool single = end && size == 1 && lrel && end_rel;
        const bool clus = end && !single;
        const unsigned ms = __ballot_sync(FULL_MASK, single);
        const unsigned mc = __ballot_sync(FULL_MASK, clus);
        int sbase = 0, cbase = 0, ovf = 0;
        long long pbase = 0;
        if (lane == 0) {
            if (ms) sbase = atomicAdd(&ctr->nsingle, __popc(ms));
            if (mc) {
                pbase = atomicAdd((unsigned long long *)&ctr->pool_need,
                                  (unsigned long long)(rep_size(nb) * __popc(mc)));
                // a fixed pool (graph-captured level loop) that cannot hold these
                // representations: the level is flagged and the clusters are dropped (their
                // columns belong to no node and are left alone; the levels are redone)
                ovf = pool_cap > 0 && pbase + rep_size(nb) * __popc(mc) > pool_cap;
                if (ovf) atomicOr(&ctr->overflow, 1);
                else cbase = atomicAdd(&ctr->ncluster, __popc(mc));
            }
        }
        sbase = __shfl_sync(FULL_MASK, sbase, 0);
        cbase = __shfl_sync(FULL_MASK, cbase, 0);
        pbase = __shfl_sync(FULL_MASK, pbase, 0);
        ovf = __shfl_sync(FULL_MASK, ovf, 0);
        const bool emit = clus && !ovf;
        // reserve next-level active-list slots for the cluster columns (warp prefix sum)
        int csz = emit ? size : 0, incl = csz;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        const int ctot = __shfl_sync(FULL_MASK, incl, 31);
        int abase = 0;
        if (lane == 0 && ctot) abase = atomicAdd(&ctr->nactive, ctot);
        abase = __shfl_sync(FULL_MASK, abase, 0);
        const unsigned below = (1u << lane) - 1u;
        if (single) {
            SingleItem it;
            it.col = c;
            it.node = w;
            singles[sbase + __popc(ms & below)] = it;
        }
        if (emit) {
            const int k = __popc(mc & below);
            ClusterItem it;
            it.node = w;
            it.c0 = gs;
            it.c1 = c;
            it.act = abase + incl - csz;
            it.lnb = (gs > N.c0) ? hi[gs - 1] : N.lnb;
            it.rnb = (c < N.c1) ? ln : N.rnb;
            clusters[cbase + k] = it;
            cluster_rep[cbase + k] = pbase + rep_size(nb) * k;
            maxsize = max(maxsize, size);
            nclus++;
        }
        if (mask) {
            const int b = 31 - __clz(mask);
            gstart = base + b + 1;
            gstart_rel = (mrel >> b) & 1u;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        maxsize = max(maxsize, __shfl_xor_sync(FULL_MASK, maxsize, o));
        nclus += __shfl_xor_sync(FULL_MASK, nclus, o);
    }
    if (lane == 0 && nclus) {
        atomicMax(&ctr->maxcluster, maxsize);
        atomicMax(&info->largest, maxsize);
        atomicAdd(&info->nclusters, nclus);
        atomicMax(&info->dmax, N.depth + 1);
    }
}

__global__ void k_classify(int nnode, const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                           const double *__restrict__ lo, const double *__restrict__ hi,
                           double gaptol, double absfac, double *gapl, double *gapr,
                           SingleItem *singles,
                           ClusterItem *clusters, long long *cluster_rep, int *cnode,
                           LevelCounters *ctr, DevInfo *info, const int *dnnode,
                           long long pool_cap) {
    // one warp per item; a grid smaller than the items loops over them
    const int nw_ = gridDim.x * (blockDim.x >> 5);
    const int bound_ = (dnnode ? *dnnode : nnode);
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < bound_; w += nw_)
        k_classify_item(w, nnode, nodes, blks, lo, hi, gaptol, absfac, gapl, gapr, singles, clusters,
                        cluster_rep, cnode, ctr, info, dnnode, pool_cap);
}

void launch_classify(int nnode, const Node *nodes, const BlkDesc *blks, const double *lo,
                     const double *hi, double gaptol, double absfac, double *gapl, double *gapr,
                     SingleItem *singles, ClusterItem *clusters, long long *cluster_rep,
                     int *cnode, LevelCounters *ctr, DevInfo *info, cudaStream_t s,
                     const int *dnnode, long long pool_cap) {
    if (nnode <= 0) return;
    const int wpb = 4;
    // with a device count the grid loops over the nodes
    const unsigned grid = dnnode ? (unsigned)std::min((nnode + wpb - 1) / wpb, 152 * 8)
                                 : (unsigned)((nnode + wpb - 1) / wpb);
    k_classify<<<grid, 32 * wpb, 0, s>>>(nnode, nodes, blks, lo, hi, gaptol,
                                                            absfac, gapl, gapr, singles, clusters,
                                                            cluster_rep, cnode, ctr, info, dnnode,
                                                            pool_cap);
}

// ------------------------------------------------------------------ cluster ends

// Alg. "Shifting the spectrum", first step: refine the extreme eigenvalues of every cluster
// before the shift.  A group of E lanes owns one end (group 2c: lambda_p, group 2c+1:
// lambda_q of cluster c) and multisects it until the interval is below 1e-3 of a lower
// bound on the gap to the inner neighbour (so that a shift just outside the interval
// leaves that end well separated in the child) or at full accuracy (4 eps |lambda|).  The
// bound starts from the neighbour's interval and tightens with every sample whose count
// shows the neighbour on its far side.  Two launches: phase 0 counts in double-float and
// stops at 1e-13 relative width (near the practical accuracy of its counts on the scaled
// copy), phase 1 checks those bounds with binary64 counts, widens where they fail, and
// continues in binary64 with fewer lanes per end (the binary64 pipe, not latency, bounds
// it when ends are many).  A cluster of one member (cut out by the absolute-gap split) has
// no inner neighbour: the group of its left end refines its one eigenvalue below 1e-3 of
// the smaller gap to its outer neighbours (so that the shift next to it leaves it with a
// relative gap of about 1e3 in the child), and the group of its right end stays idle.
__device__ __forceinline__ void k_refine_ends_item(long long tid, int E, int ncluster,
                              const ClusterItem *__restrict__ clusters,
                              const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                              const double *__restrict__ pool, const int *__restrict__ jloc,
                              double *lo, double *hi, int E_host, int phase, double2 *carry,
                              DevInfo *info, const int *dncluster) {
    const int lane = threadIdx.x & 31;
    const int g = tid / E, k = lane % E, gbase = lane - k;
    const unsigned gmask = (E == 32) ? 0xffffffffu : (((1u << E) - 1u) << gbase);
    bool active = g < 2 * ncluster;
    const int side = g & 1;
    int n = 1, tgt = 1, col = 0;
    Node P;
    P.dfok = 0;
    const double *pd = pool;
    double L = 0.0, H = 0.0, nb = 0.0;
    if (active && side == 1 && clusters[g >> 1].c0 == clusters[g >> 1].c1) active = false;
    if (active) {
        const ClusterItem C = clusters[g >> 1];
        P = nodes[C.node];
        n = blks[P.blk].n;
        pd = pool + P.rep;
        col = side ? C.c1 : C.c0;
        tgt = jloc[col];
        L = lo[col];
        H = hi[col];
        if (C.c0 == C.c1) {
            // a lower bound on the right neighbour that also bounds the gap to the left one:
            // the bisection tolerance then follows min(left gap, right gap)
            const double gmin = fmin(L - C.lnb, C.rnb - H);
            nb = (gmin > 0.0 && gmin < INFINITY) ? H + gmin : -INFINITY;
        } else {
            nb = side ? hi[col - 1] : lo[col + 1];
        }
        // phase 1 resumes with the neighbour bound phase 0 tightened
        if (phase == 1) nb = carry[g].x;
    }
    unsigned long long steps = 0;
    if (phase == 1) {
        // the double-float phase's bounds hold for its perturbed copy of the representation:
        // verify them with binary64 counts and widen by that copy's error bound if needed
        const double kap = 32.0 * n * 0x1p-47;
        for (int attempt = 0; attempt < 6; ++attempt) {
            int okL = 1, okH = 1;
            if (active) {
                if (E >= 2) {
                    int cnt = 0;
                    if (k < 2) { cnt = negcount_ldl(n, pd, pd + 2 * n, k == 0 ? L : H); steps += n; }
                    okL = __shfl_sync(gmask, cnt, gbase) < tgt;
                    okH = __shfl_sync(gmask, cnt, gbase + 1) >= tgt;
                } else {
                    okL = negcount_ldl(n, pd, pd + 2 * n, L) < tgt;
                    okH = negcount_ldl(n, pd, pd + 2 * n, H) >= tgt;
                    steps += 2ull * n;
                }
            } else if (E >= 2) {
                (void)__shfl_sync(gmask, 0, gbase);
                (void)__shfl_sync(gmask, 0, gbase + 1);
            }
            const bool ok = okL && okH;
            if (__all_sync(0xffffffffu, ok || !active)) break;
            if (active && !ok) {
                // geometric from the interval's own width up to the copy's error bound
                // kap (16^attempt), then beyond it
                const double w0 = fmax(H - L, kEps * fmax(fabs(L), fabs(H)));
                const double f = fmin(ldexp(w0, 4 * (attempt + 1)),
                                      ldexp(kap, 4 * attempt) * fmax(fmax(fabs(L), fabs(H)), kSafmin));
                if (!okL) L -= f;
                if (!okH) H += f;
            }
        }
    }
    int sw = 0, rounds = 0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double w = H - L;
        const double gap_lb = side ? (L - nb) : (nb - H);
        double tol = fmax(4.0 * kEps * fmax(fabs(L), fabs(H)), 1e-3 * fmax(gap_lb, 0.0));
        if (phase == 0) tol = fmax(tol, kRefineDfRtol * fmax(fabs(L), fabs(H)));
        bool done = !active || !(w > tol);
        const double x = L + (k + 1) * (w / (E + 1));
        if (__ballot_sync(0xffffffffu, !(x > L && x < H)) & gmask) done = true;
        if (__all_sync(0xffffffffu, done)) break;
        int cnt = 0;
        if (!done) {
            cnt = (phase == 0) ? node_count(P, n, pd, x) : negcount_ldl(n, pd, pd + 2 * n, x);
            steps += n;
            ++sw;
        }
        ++rounds;
        const unsigned bal = __ballot_sync(0xffffffffu, cnt < tgt);
        const int t = __popc(bal & gmask);
        const double xl = __shfl_sync(0xffffffffu, x, gbase + (t > 0 ? t - 1 : 0));
        const double xh = __shfl_sync(0xffffffffu, x, gbase + (t < E ? t : E - 1));
        // left end: count <= j gives lambda_{j+1} >= x (largest such x); right end:
        // count >= j - 1 gives lambda_{j-1} < x (smallest such x)
        const bool nbl = side ? (cnt >= tgt - 1) : (cnt <= tgt);
        const unsigned hb = (__ballot_sync(0xffffffffu, nbl && !done) & gmask) >> gbase;
        const int first = hb ? __ffs(hb) - 1 : 0, last = hb ? 31 - __clz(hb) : 0;
        const double xf = __shfl_sync(0xffffffffu, x, gbase + first);
        const double xlst = __shfl_sync(0xffffffffu, x, gbase + last);
        if (!done) {
            if (hb) nb = side ? fmin(nb, xf) : fmax(nb, xlst);
            if (t > 0) L = xl;
            if (t < E) H = xh;
        }
    }
    if (info->trace) trace_sweeps(info, 1 + phase, active && k == 0, sw, rounds);
    if (active && k == 0) {
        lo[col] = L;
        hi[col] = H;
        if (phase == 0) carry[g] = make_double2(nb, 0.0);
    }
    for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, o);
    if (lane == 0 && steps) atomicAdd(&info->shift_steps, steps);
}

__global__ void k_refine_ends(int ncluster, const ClusterItem *__restrict__ clusters,
                              const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                              const double *__restrict__ pool, const int *__restrict__ jloc,
                              double *lo, double *hi, int E_host, int phase, double2 *carry,
                              DevInfo *info, const int *dncluster) {
    // with a device count the lanes per end follow the same rule the host applies, and a
    // grid smaller than the ends' lanes loops over them one warp (whole groups) at a time
    if (dncluster) ncluster = *dncluster;
    const int E = dncluster ? refine_lanes(2ll * ncluster, phase) : E_host;
    const long long total = 2ll * ncluster * E;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (long long wb = first; wb < total; wb += stride)
        k_refine_ends_item(wb + (threadIdx.x & 31), E, ncluster, clusters, nodes, blks, pool, jloc, lo, hi, E_host, phase, carry, info, dncluster);
}

void launch_refine_ends(int ncluster, const ClusterItem *clusters, const Node *nodes,
                        const BlkDesc *blks, const double *pool, const int *jloc, double *lo,
                        double *hi, double2 *carry, DevInfo *info, cudaStream_t s,
                        const int *dncluster) {
    if (ncluster <= 0) return;
    // lanes per end: many ends -> fewer lanes (throughput), few ends -> more (latency)
    const long long ends = 2ll * ncluster;
    for (int phase = 0; phase < 2; ++phase) {
        const int E = refine_lanes(ends, phase);
        // with a device count (at most ncluster) the grid loops: up to 64 warps per SM
        const long long threads =
            dncluster ? std::min(std::max(refine_lane_cap(phase), ends * (phase == 0 ? 4 : 1)),
                                 152ll * 2048)
                      : ends * E;
        const int bs = threads >= 152ll * 64 * 2 ? 64 : 32; // small launches spread over the SMs
        k_refine_ends<<<(unsigned)((threads + bs - 1) / bs), bs, 0, s>>>(
            ncluster, clusters, nodes, blks, pool, jloc, lo, hi, E, phase, carry, info, dncluster);
    }
}

// ------------------------------------------------------------------ cluster shift

// Trial dstqds L+ D+ L+^T = L D L^T - tau I in homogeneous form (see negcount_ldl).
// Existence: no exact zero pivot and finite values.  Element growth: max |d+_i|, the
// division c_i / c_{i-1} being off the recurrence's critical path.  With STORE, the
// unscaled c_i go to U[i] and the power-of-two rescale applied after step i to K[i].
// As in negcount_ldl the loop runs in blocks of 8 steps without a data-dependent branch
// and normalises (a, c) at the end of a block (K[i] is nonzero only there); a block in
// which some c was zero or left [2^-400, 2^400] is redone with the per-step rules.

// One step with the per-step rules.
template <bool STORE>
__device__ __forceinline__ void trial_step_exact(int i, bool last, double di, double li, double tau,
                                                 double *U, int *K, int kstride, double &a,
                                                 double &cp, bool &zero, double &gn, double &gd) {
    double c = fma(di, cp, a);
    const bool z = is_zero(c);
    zero |= z;
    c = z ? -cp * 0x1p-80 : c;
    const double ac = fabs(c), acp = fabs(cp);
    const bool up = ac * gd > gn * acp;
    gn = up ? ac : gn;
    gd = up ? acp : gd;
    int k = 0;
    if (!last) {
        a = fma(-tau, c, li * a);
        if (STORE) U[i] = c;
        const int ex = biased_exp(c);
        if ((unsigned)(ex - (1023 - 200)) > 400u) {
            k = 1023 - ex;
            const double sc = pow2i(k);
            c *= sc;
            a *= sc;
        }
    } else if (STORE) {
        U[i] = c;
    }
    if (STORE) K[(size_t)i * kstride] = k;
    cp = c;
}

template <bool STORE>
__device__ void trial_shift(int n, const double *__restrict__ d, const double *__restrict__ dll,
                            double tau, double *U, int *K, int kstride, bool &exists,
                            double &growth) {
    double a = -tau, cp = 1.0;
    bool zero = false;
    // running maximum of |c_i / c_{i-1}| kept as a fraction gn / gd: no division on the
    // recurrence's critical path (non-finite values propagate and are caught at the end)
    double gn = 0.0, gd = 1.0;
    // operands of step i + 1 are loaded while step i runs (software prefetch)
    double dn = __ldg(d), ln = (n > 1) ? __ldg(dll) : 0.0;
    int i = 0;
    for (; i + 8 < n; i += 8) {
        const double a0 = a, c0 = cp, gn0 = gn, gd0 = gd;
        bool bad = false;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double di = dn, li = ln;
            dn = __ldg(d + i + u + 1);
            ln = (i + u + 1 < n - 1) ? __ldg(dll + i + u + 1) : 0.0;
            const double c = fma(di, cp, a);
            // zero, or outside [2^-400, 2^400] (the growth test multiplies two values)
            bad |= (unsigned)(biased_exp(c) - (1023 - 400)) > 800u;
            const double ac = fabs(c), acp = fabs(cp);
            const bool up = ac * gd > gn * acp;
            gn = up ? ac : gn;
            gd = up ? acp : gd;
            a = fma(-tau, c, li * a);
            if (STORE) {
                U[i + u] = c;
                K[(size_t)(i + u) * kstride] = 0;
            }
            cp = c;
        }
        const int ex = biased_exp(cp), ea = biased_exp(a);
        if (__builtin_expect(bad || ea == 0x7ff, 0)) {
            a = a0;
            cp = c0;
            gn = gn0;
            gd = gd0;
            for (int k = i; k < i + 8; ++k)
                trial_step_exact<STORE>(k, false, __ldg(d + k), __ldg(dll + k), tau, U, K, kstride,
                                        a, cp, zero, gn, gd);
        } else {
            const int k = 1023 - ex;
            const double q = pow2i(k);
            cp *= q;
            a *= q;
            if (STORE) K[(size_t)(i + 7) * kstride] = k;
        }
    }
    for (; i < n; ++i) {
        const double di = dn, li = ln;
        if (i + 1 < n) {
            dn = __ldg(d + i + 1);
            ln = (i + 1 < n - 1) ? __ldg(dll + i + 1) : 0.0;
        }
        trial_step_exact<STORE>(i, i == n - 1, di, li, tau, U, K, kstride, a, cp, zero, gn, gd);
    }
    const double g = gn / gd;
    exists = is_finite(tau) && !zero && is_finite(g) && is_finite(cp) && is_finite(a);
    growth = exists ? g : INFINITY;
}

// Backward progressive recurrence of L D L^T - tau I (Alg. dqds): p_{n-1} = d_{n-1} - tau,
// p_k = d_k p_{k+1} / (p_{k+1} + dll_k) - tau, in homogeneous form p = N / M with no
// division on the chain:  M_k = N + dll_k M,  N_k = (d_k - tau) N - (tau dll_k) M,
// rescaled by a power of two every eight steps (an overflow inside a block gives a
// non-finite value, which the envelope test treats as a failure).  Stores N_k, M_k.
__device__ void dqds_backward_store(int n, const double *__restrict__ d,
                                    const double *__restrict__ dll, double tau, double *Ns,
                                    double *Ms) {
    double N = __ldg(d + n - 1) - tau, M = 1.0;
    Ns[n - 1] = N;
    Ms[n - 1] = M;
    int k = n - 2;
    for (; k >= 7; k -= 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double dk = __ldg(d + k - u), lk = __ldg(dll + k - u);
            const double Mk = fma(lk, M, N);
            N = fma(dk - tau, N, -(tau * lk) * M);
            M = Mk;
            Ns[k - u] = N;
            Ms[k - u] = M;
        }
        const int ex = biased_exp(M);
        const double sc = (ex > 0 && ex < 0x7ff) ? pow2i(1023 - ex) : 1.0;
        N *= sc;
        M *= sc;
    }
    for (; k >= 0; --k) {
        const double dk = __ldg(d + k), lk = __ldg(dll + k);
        const double Mk = fma(lk, M, N);
        N = fma(dk - tau, N, -(tau * lk) * M);
        M = Mk;
        Ns[k] = N;
        Ms[k] = M;
    }
}

// The first two candidates of every cluster, one lane each (16 clusters per warp):
// tau_l = lo_p - 100 eps |lo_p| on even lanes, tau_r = hi_q + 100 eps |hi_q| on odd lanes.
// Each stores its c_i and rescale exponents in the child's slots (tau_l: d, tau_r: dl;
// exponents interleaved in dll) for the conversion, and its existence and growth in
// tri[2 ci + side].
__global__ void k_shift_trials(int ncluster, const ClusterItem *__restrict__ clusters,
                               const long long *__restrict__ cluster_rep,
                               const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                               const double *__restrict__ pool, double *childpool,
                               const double *__restrict__ lo, const double *__restrict__ hi,
                               unsigned fault_mask, double2 *tri, DevInfo *info,
                               const int *dncluster) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int ci = t >> 1, side = t & 1;
    unsigned long long steps = 0;
    if (dncluster) ncluster = *dncluster;
    if (ci < ncluster) {
        const ClusterItem C = clusters[ci];
        const Node P = nodes[C.node];
        const int n = blks[P.blk].n;
        const double *pd = pool + P.rep;
        double *cd = childpool + cluster_rep[ci];
        const double Lp = lo[C.c0], Hq = hi[C.c1];
        double tau = side ? Hq + MR3_TAU_OFFSET * kEps * fabs(Hq) : Lp - MR3_TAU_OFFSET * kEps * fabs(Lp);
        if (side == 0 && (fault_mask & MR3_FAULT_NAN_SHIFT)) tau = NAN;
        bool ex = false;
        double g = INFINITY;
        trial_shift<true>(n, pd, pd + 2 * n, tau, side ? cd + n : cd, (int *)(cd + 2 * n) + side, 2,
                    ex, g);
        tri[2 * ci + side] = make_double2(ex ? 1.0 : 0.0, g);
        steps = n;
    }
    for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(FULL_MASK, steps, o);
    if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&info->shift_steps, steps);
}

// The shift decision of one cluster: its tau, which stored factorization holds the child
// (0: tau_l's, 1: tau_r's, 2: recomputed), and whether it was accepted untested.
struct ShiftDecision {
    double tau;
    int win;
    int untested;
};

// Candidates of a cluster: tau_l0, tau_r0 at 100 eps from the refined ends, the back-off
// unit delta = max(100 eps |lambda|, 1e-3 W) and the growth threshold 8 spdiam(M_root).
struct ShiftSetup {
    double tau_l0, tau_r0, delta, thresh;
};
__device__ __forceinline__ ShiftSetup shift_setup(const ClusterItem &C, const BlkDesc &B,
                                                  const double *__restrict__ lo,
                                                  const double *__restrict__ hi) {
    const double Lp = lo[C.c0], Hq = hi[C.c1];
    ShiftSetup S;
    S.tau_l0 = Lp - MR3_TAU_OFFSET * kEps * fabs(Lp);
    S.tau_r0 = Hq + MR3_TAU_OFFSET * kEps * fabs(Hq);
    S.delta = fmax(100.0 * kEps * fmax(fabs(Lp), fabs(Hq)), 1e-3 * (Hq - Lp));
    S.thresh = 8.0 * B.spdiam;
    return S;
}

// Clusters per launch from which the envelope test runs before the back-off ladder
// (throughput regime) instead of beside it (latency regime): four warps per SM.
constexpr int kEnvSequentialClusters = 152 * 32 * 4;

__host__ __device__ __forceinline__ int ladder_width(int max_tries) {
    return 2 * (max(2, min(max_tries, 16)) - 1);
}

// The "more sophisticated test" of Alg. "Shifting the spectrum" (remark 3), for the
// clusters whose first candidates failed the plain growth test: element growth is
// harmless where every eigenvector of the cluster is small, so the growth of a first
// candidate is weighed by a bound on the envelope of the cluster's invariant subspace,
// env2(k) = sum_{j in cluster} z_j(k)^2.  With mu_j = lambda_j - tau the child's
// eigenvalues and gamma_k the twist element of L D L^T - tau I at k (Alg. Getvec:
// gamma_k = s_k + p_k + tau from the forward and backward recurrences),
//   1 / gamma_k = [(L D L^T - tau I)^{-1}]_kk = sum_j z_j(k)^2 / mu_j;
// the cluster's mu_j share one sign (tau lies outside the cluster) and are at most Lambda
// in magnitude (the cluster's far end seen from tau), every other |mu_j| is at least g
// (the distance from tau to the nearest eigenvalue outside the cluster), so
//   env2(k) <= Lambda (1 / |gamma_k| + 1 / g)   (capped at 1).
// The candidate passes when
//   max_k ( |d+_k| env2(k) + |dll+_k| env2(k+1) ) <= 8 spdiam(M_root),
// the plain test's threshold applied to the z-weighted pivots of z^T L+ |D+| L+^T z.
// Over the clusters queued by k_shift_select (threads past the queue's length return):
// shift_envback, one lane per first candidate in warps of their own inside the back-off
// ladder's launch (the two chains of n steps run side by side), runs the backward
// recurrence (N, M of tau_l at [3n, 5n) of the child's slot, of tau_r at [5n, 7n));
// k_shift_envtest, one warp per cluster with the indices split over the lanes, forms
// s_k = d+_k - d_k from the trial's stored c_k and p_k = N_k / M_k, reduces the weighted
// growth, and takes the better passing candidate, which k_shift_pick then keeps over the
// ladder.  The test needs magnitudes only: its divisions use the hardware's approximate
// reciprocal (rcp.approx.ftz.f64); and since env2 <= 1, an index whose |d+_k| + |dll+_k|
// is below the threshold cannot fail it, so the envelope is formed only around the others.
__device__ unsigned long long shift_envback(long long t, int nslots,
                                            const ClusterItem *__restrict__ clusters,
                                            const long long *__restrict__ cluster_rep,
                                            const Node *__restrict__ nodes,
                                            const BlkDesc *__restrict__ blks,
                                            const double *__restrict__ pool, double *childpool,
                                            const double *__restrict__ lo,
                                            const double *__restrict__ hi,
                                            const double2 *__restrict__ tri, unsigned fault_mask,
                                            const int *__restrict__ ladder,
                                            const int *__restrict__ counts) {
    const int li = (int)(t >> 1), side = (int)(t & 1);
    unsigned long long steps = 0;
    if (li < nslots && li < counts[0]) {
        const int ci = ladder[li];
        if (tri[2 * ci + side].x != 0.0) {
            const ClusterItem C = clusters[ci];
            const Node P = nodes[C.node];
            const int n = blks[P.blk].n;
            const double *pd = pool + P.rep;
            double *Ns = childpool + cluster_rep[ci] + 3ll * n + 2ll * n * side;
            const double Lp = lo[C.c0], Hq = hi[C.c1];
            double tau = side ? Hq + MR3_TAU_OFFSET * kEps * fabs(Hq)
                              : Lp - MR3_TAU_OFFSET * kEps * fabs(Lp);
            if (side == 0 && (fault_mask & MR3_FAULT_NAN_SHIFT)) tau = NAN;
            dqds_backward_store(n, pd, pd + 2 * n, tau, Ns, Ns + n);
            steps = n;
        }
    }
    return steps;
}

__device__ __forceinline__ void k_shift_envtest_item(int li, int nslots, const ClusterItem *__restrict__ clusters,
                                const long long *__restrict__ cluster_rep,
                                const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                                const double *__restrict__ pool,
                                const double *__restrict__ childpool,
                                const double *__restrict__ lo, const double *__restrict__ hi,
                                const double2 *__restrict__ tri, unsigned fault_mask,
                                const int *__restrict__ ladder, const int *__restrict__ counts,
                                ShiftDecision *dec, DevInfo *info) {
    const int lane = threadIdx.x & 31;
    if (fault_mask & MR3_FAULT_SHIFT_REJECT) return;
    const int ci = ladder[li];
    const ClusterItem C = clusters[ci];
    const Node P = nodes[C.node];
    const int n = blks[P.blk].n;
    const double *pd = pool + P.rep, *pdl = pd + n;
    const double *cd = childpool + cluster_rep[ci];
    const double Lp = lo[C.c0], Hq = hi[C.c1];
    double wside[2] = {INFINITY, INFINITY};
    for (int side = 0; side < 2; ++side) {
        double tau = side ? Hq + MR3_TAU_OFFSET * kEps * fabs(Hq) : Lp - MR3_TAU_OFFSET * kEps * fabs(Lp);
        if (side == 0 && (fault_mask & MR3_FAULT_NAN_SHIFT)) tau = NAN;
        const double Lam = side ? tau - Lp : Hq - tau;
        const double g = fmin(tau - C.lnb, C.rnb - tau);
        if (tri[2 * ci + side].x == 0.0 || !(g > 0.0) || !(Lam > 0.0)) continue;
        const double ig = 1.0 / g;
        const double *U = side ? cd + n : cd;
        const int *K = (const int *)(cd + 2 * n) + side;
        const double *Ns = cd + 3ll * n + 2ll * n * side, *Ms = Ns + n;
        // d+_k = U[k] / U[k-1] 2^-K[k-1] (U[-1] = 1, K[-1] = 0); env2 bound at k
        auto dplus = [&](int k) {
            const double um = (k > 0) ? U[k - 1] : 1.0;
            const int km = (k > 0) ? K[2 * (k - 1)] : 0;
            return U[k] * rcp_approx(um) * pow2i(-km);
        };
        auto env_at = [&](int k, double dk) {
            const double gam = (dk - pd[k]) + Ns[k] * rcp_approx(Ms[k]) + tau;
            return fmin(1.0, Lam * (fabs(rcp_approx(gam)) + ig));
        };
        // term_k <= |d+_k| + |dll+_k| (env2 <= 1): only the indices where that sum exceeds
        // the threshold need the envelope (theirs and the next one's)
        const double thr = 8.0 * blks[P.blk].spdiam;
        double wg = 0.0;
        bool carry_need = false; // the previous chunk's last index needs env2 of this chunk's first
        for (int base = 0; base < n; base += 32) {
            const int k = base + lane;
            double dk = 0.0, dllk = 0.0;
            if (k < n) {
                dk = dplus(k);
                if (k < n - 1) {
                    const double dl = pdl[k];
                    dllk = fabs(dl * dl * rcp_approx(dk));
                }
            }
            const double mag = fabs(dk) + dllk;
            const bool need = (k < n) && !(mag <= thr);
            const bool need_prev_raw = __shfl_up_sync(FULL_MASK, need && dllk != 0.0, 1);
            const bool need_prev = (lane == 0) ? carry_need : need_prev_raw;
            carry_need = __shfl_sync(FULL_MASK, need && dllk != 0.0, 31);
            double env = 0.0;
            if (k < n && (need || need_prev)) env = env_at(k, dk);
            double env_next = __shfl_down_sync(FULL_MASK, env, 1);
            if (lane == 31 && need && dllk != 0.0 && k + 1 < n) env_next = env_at(k + 1, dplus(k + 1));
            if (need) {
                const double term = fabs(dk) * env + dllk * env_next;
                wg = (term > wg || term != term) ? term : wg;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_xor_sync(FULL_MASK, wg, o);
            wg = (v > wg || v != v) ? v : wg;
        }
        wside[side] = (wg == wg) ? wg : INFINITY;
    }
    if (lane == 0) {
        const ShiftSetup S = shift_setup(C, blks[P.blk], lo, hi);
        const bool v0 = wside[0] <= S.thresh, v1 = wside[1] <= S.thresh;
        if (v0 || v1) {
            const int se = (v0 && (!v1 || wside[0] <= wside[1])) ? 0 : 1;
            dec[ci] = {se ? S.tau_r0 : S.tau_l0, se, 0};
            atomicAdd(&info->env_accepted, 1);
        }
    }
}

__global__ void k_shift_envtest(int nslots, const ClusterItem *__restrict__ clusters,
                                const long long *__restrict__ cluster_rep,
                                const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                                const double *__restrict__ pool,
                                const double *__restrict__ childpool,
                                const double *__restrict__ lo, const double *__restrict__ hi,
                                const double2 *__restrict__ tri, unsigned fault_mask,
                                const int *__restrict__ ladder, const int *__restrict__ counts,
                                ShiftDecision *dec, DevInfo *info) {
    // one warp per queued cluster; a grid smaller than the queue loops over it
    const int nw_ = gridDim.x * (blockDim.x >> 5);
    const int bound_ = min(nslots, counts[0]);
    for (int li = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); li < bound_; li += nw_)
        k_shift_envtest_item(li, nslots, clusters, cluster_rep, nodes, blks, pool, childpool, lo,
                             hi, tri, fault_mask, ladder, counts, dec, info);
}

// One thread per cluster: take the better existing first candidate if its growth passes,
// else queue the cluster for the envelope test and the back-off ladder.
__global__ void k_shift_select(int ncluster, const ClusterItem *__restrict__ clusters,
                               const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                               const double *__restrict__ lo, const double *__restrict__ hi,
                               unsigned fault_mask, const double2 *__restrict__ tri,
                               ShiftDecision *dec, int *ladder, int *counts, DevInfo *info,
                               const int *dncluster) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= (dncluster ? *dncluster : ncluster)) return;
    const ClusterItem C = clusters[ci];
    const BlkDesc B = blks[nodes[C.node].blk];
    const ShiftSetup S = shift_setup(C, B, lo, hi);
    const double2 t0 = tri[2 * ci], t1 = tri[2 * ci + 1];
    const bool e0 = t0.x != 0.0, e1 = t1.x != 0.0;
    int sel = -1;
    if (e0 && e1) sel = (t0.y <= t1.y) ? 0 : 1;
    else if (e0) sel = 0;
    else if (e1) sel = 1;
    const bool reject_all = (fault_mask & MR3_FAULT_SHIFT_REJECT) != 0;
    if (sel >= 0 && !reject_all && (sel == 0 ? t0.y : t1.y) <= S.thresh) {
        dec[ci] = {sel == 0 ? S.tau_l0 : S.tau_r0, sel, 0};
    } else {
        dec[ci] = {0.0, -1, 0};
        ladder[atomicAdd(counts, 1)] = ci;
        atomicAdd(&info->ladder, 1);
    }
}

// One lane per back-off candidate: tau_l0 - 2^(t-1) delta (even j) and
// tau_r0 + 2^(t-1) delta (odd j), t = j / 2 + 1, for every queued cluster that the
// envelope test did not settle.
// Blocks from ladder_blocks on run shift_envback instead.
__global__ void k_shift_ladder(int nslots, int max_tries, const ClusterItem *__restrict__ clusters,
                               const long long *__restrict__ cluster_rep,
                               const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                               const double *__restrict__ pool, double *childpool,
                               const double *__restrict__ lo, const double *__restrict__ hi,
                               const double2 *__restrict__ tri, unsigned fault_mask,
                               const int *__restrict__ ladder, const int *__restrict__ counts,
                               const ShiftDecision *__restrict__ dec, double2 *lad,
                               unsigned ladder_blocks, DevInfo *info, int regime,
                               const int *dncluster) {
    // blocks [0, ladder_blocks) take back-off candidates, the others backward recurrences;
    // a grid smaller than its role's work loops over it.  With a device count (regime 1:
    // the launch of the few-clusters order, 2: of the many-clusters order) the launch runs
    // only when the count selects its order.
    if (regime != 0) {
        const bool many = *dncluster >= kEnvSequentialClusters;
        if ((regime == 1) == many) return;
    }
    const bool env_role = blockIdx.x >= ladder_blocks;
    const long long rb = env_role ? blockIdx.x - ladder_blocks : blockIdx.x;
    const long long nrb = env_role ? gridDim.x - ladder_blocks : ladder_blocks;
    const int NL = ladder_width(max_tries);
    const int nq = min(nslots, counts[0]);
    const long long total = env_role ? 2ll * nq : (long long)nq * NL;
    unsigned long long steps = 0;
    for (long long base = rb * blockDim.x; base < total; base += nrb * blockDim.x) {
        const long long gid = base + threadIdx.x;
        if (env_role) {
            steps += shift_envback(gid, nslots, clusters, cluster_rep, nodes, blks, pool,
                                   childpool, lo, hi, tri, fault_mask, ladder, counts);
            continue;
        }
        const int li = (int)(gid / NL), j = (int)(gid % NL);
        if (li < nq && dec[ladder[li]].win < 0) {
            const int ci = ladder[li];
            const ClusterItem C = clusters[ci];
            const Node P = nodes[C.node];
            const BlkDesc B = blks[P.blk];
            const int n = B.n;
            const ShiftSetup S = shift_setup(C, B, lo, hi);
            const double off = ldexp(S.delta, j / 2);
            const double tau = (j & 1) ? S.tau_r0 + off : S.tau_l0 - off;
            const double *pd = pool + P.rep;
            bool ex = false;
            double g = INFINITY;
            trial_shift<false>(n, pd, pd + 2 * n, tau, nullptr, nullptr, 0, ex, g);
            lad[(long long)li * NL + j] = make_double2(ex ? 1.0 : 0.0, g);
            steps += n;
        }
    }
    for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(FULL_MASK, steps, o);
    if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&info->shift_steps, steps);
}

// One thread per queued cluster: the first back-off step t whose better existing candidate
// passes the growth test wins (recomputed); else the least growth over every candidate,
// the first two included, accepted untested.
__global__ void k_shift_pick(int nslots, int max_tries, unsigned fault_mask,
                             const ClusterItem *__restrict__ clusters,
                             const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                             const double *__restrict__ lo, const double *__restrict__ hi,
                             const double2 *__restrict__ tri, const int *__restrict__ ladder,
                             int *counts, const double2 *__restrict__ lad, ShiftDecision *dec,
                             int *recomp, DevInfo *info) {
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nslots || li >= counts[0]) return;
    const int NL = ladder_width(max_tries);
    const int ci = ladder[li];
    if (dec[ci].win >= 0) return; // settled by the envelope test
    const ClusterItem C = clusters[ci];
    const ShiftSetup S = shift_setup(C, blks[nodes[C.node].blk], lo, hi);
    const bool reject_all = (fault_mask & MR3_FAULT_SHIFT_REJECT) != 0;
    const double2 *L = lad + (long long)li * NL;
    auto tau_of = [&](int j) {
        const double off = ldexp(S.delta, j / 2);
        return (j & 1) ? S.tau_r0 + off : S.tau_l0 - off;
    };
    ShiftDecision D = {0.0, -1, 0};
    for (int jL = 0; jL < NL; jL += 2) {
        const bool exL = L[jL].x != 0.0, exR = L[jL + 1].x != 0.0;
        int sel = -1;
        if (exL && exR) sel = (L[jL].y <= L[jL + 1].y) ? jL : jL + 1;
        else if (exL) sel = jL;
        else if (exR) sel = jL + 1;
        if (sel >= 0 && !reject_all && L[sel].y <= S.thresh) { D = {tau_of(sel), 2, 0}; break; }
    }
    if (D.win < 0) {
        const double2 t0 = tri[2 * ci], t1 = tri[2 * ci + 1];
        const bool e0 = t0.x != 0.0, e1 = t1.x != 0.0;
        double gb = INFINITY;
        int jb = -1;
        for (int j = 0; j < NL; ++j)
            if (L[j].x != 0.0 && L[j].y < gb) { gb = L[j].y; jb = j; }
        if (e0 && t0.y <= gb && (!e1 || t0.y <= t1.y)) D = {S.tau_l0, 0, 1};
        else if (e1 && t1.y <= gb) D = {S.tau_r0, 1, 1};
        else if (jb >= 0) D = {tau_of(jb), 2, 1};
        else D = {S.tau_l0, 0, 1}; // nothing exists: keep the first candidate (flagged)
    }
    dec[ci] = D;
    if (D.win == 2) {
        recomp[atomicAdd(counts + 1, 1)] = ci;
        if (!D.untested) atomicAdd(&info->recomputed, 1);
    }
}

// One lane per cluster whose winner is a back-off candidate: its factorization again,
// stored like a first candidate on the tau_l side.
__global__ void k_shift_recompute(int nslots, const ClusterItem *__restrict__ clusters,
                                  const long long *__restrict__ cluster_rep,
                                  const Node *__restrict__ nodes, const BlkDesc *__restrict__ blks,
                                  const double *__restrict__ pool, double *childpool,
                                  const int *__restrict__ recomp, const int *__restrict__ counts,
                                  const ShiftDecision *__restrict__ dec, DevInfo *info) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long steps = 0;
    if (r < nslots && r < counts[1]) {
        const int ci = recomp[r];
        const Node P = nodes[clusters[ci].node];
        const int n = blks[P.blk].n;
        const double *pd = pool + P.rep;
        double *cd = childpool + cluster_rep[ci];
        bool ex;
        double g;
        trial_shift<true>(n, pd, pd + 2 * n, dec[ci].tau, cd, (int *)(cd + 2 * n), 2, ex, g);
        steps = n;
    }
    for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(FULL_MASK, steps, o);
    if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&info->shift_steps, steps);
}

// One warp per cluster {p..q} of node P (Alg. "Shifting the spectrum" inside a C-task).
//  1. The cluster's extreme eigenvalues come refined from k_refine_ends.
//  2. Candidates tau_l = lo_p - 100 eps |lo_p| and tau_r = hi_q + 100 eps |hi_q| (k_shift_trials,
//     one lane each; k_shift_select); a candidate exists when its factorization has no
//     zero pivot and stays finite; of
//     existing ones the smaller growth max|d+_i| is taken; it is accepted when
//     max|d+_i| <= 8 spdiam(M_root).  Otherwise back off:
//     tau_l - 2^(t-1) delta, tau_r + 2^(t-1) delta, delta = max(100 eps |lambda|, 1e-3 W)
//     (W the cluster width), t = 1 .. max_tries-1, one lane per candidate (k_shift_ladder,
//     k_shift_pick); the first t with an accepted candidate wins and is recomputed
//     (k_shift_recompute), else the least growth overall (counted untested).
//  3. The winner's c_i give the child: d+_i = c_i / c_{i-1}, l+_i = dl_i / d+_i,
//     dl+_i = d+_i l+_i, dll+_i = dl+_i l+_i, converted in place by chunks of 32.  With
//     erep the child is kept as an e-representation (Ch. 3, representation forms; Ch. 5
//     on the choice of form): its primary data are d+ and the off-diagonal entries
//     beta_i = dl_i, which dstqds leaves unchanged, so dl+ = dl exactly (every node of the
//     tree then carries the root's beta bit for bit) and dll+_i = beta_i (beta_i / d+_i).
__device__ __forceinline__ void k_shift_item(int ci, int ncluster,
                        const ClusterItem *__restrict__ clusters,
                        const long long *__restrict__ cluster_rep, const Node *__restrict__ nodes,
                        const BlkDesc *__restrict__ blks, const double *__restrict__ pool,
                        double *childpool, Node *child_nodes, double *child_tau, int *cnode,
                        int *active_list, const ShiftDecision *__restrict__ dec, int erep,
                        DevInfo *info, const int *dncluster) {
    const int lane = threadIdx.x & 31;
    const ClusterItem C = clusters[ci];
    const Node P = nodes[C.node];
    const BlkDesc B = blks[P.blk];
    const int n = B.n;
    const double *pdl = pool + P.rep + n;
    double *cd = childpool + cluster_rep[ci], *cdl = cd + n, *cdll = cd + 2 * n;
    const int p = C.c0, q = C.c1;

    // ---- 1-2. ends refined (k_refine_ends), shift chosen (k_shift_trials .. k_shift_pick)
    const ShiftDecision D = dec[ci];
    const double tau = D.tau;
    const int win = D.win;
    const bool untested = D.untested != 0;
    int *K = (int *)cdll; // int2 per element: .x candidate tau_l (or recomputed), .y tau_r

    // ---- 3. convert the stored c_i into the child representation (in place), with its
    // double-float copy for the bisection
    const double *U = (win == 1) ? cdl : cd;
    const int kofs = (win == 1) ? 1 : 0;
    double carry_u = 1.0;
    int carry_k = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const double ui = (i < n) ? U[i] : 1.0;
        const int ki = (i < n) ? K[2 * i + kofs] : 0;
        double up = __shfl_up_sync(FULL_MASK, ui, 1);
        int kp = __shfl_up_sync(FULL_MASK, ki, 1);
        if (lane == 0) { up = carry_u; kp = carry_k; }
        carry_u = __shfl_sync(FULL_MASK, ui, 31);
        carry_k = __shfl_sync(FULL_MASK, ki, 31);
        __syncwarp();
        if (i < n) {
            const double dp = (ui / up) * pow2i(-kp);
            double dllp = 0.0;
            cd[i] = dp;
            if (i < n - 1) {
                const double lp = pdl[i] / dp;
                const double dlp = erep ? pdl[i] : dp * lp;
                dllp = dlp * lp;
                cdl[i] = dlp;
                cdll[i] = dllp;
            } else {
                cdl[i] = 0.0;
                cdll[i] = 0.0;
            }
        }
        __syncwarp();
    }
    int dfexp;
    const bool dfok = df_write_copy_warp(n, cd, cdll, (float4 *)(cd + rep_df_offset(n)), dfexp);
    __syncwarp();
    build_prefix(n, cd);

    // ---- 4. child node
    for (int c = p + lane; c <= q; c += 32) {
        cnode[c] = ci;
        active_list[C.act + (c - p)] = c;
    }
    if (lane == 0) {
        Node Cn;
        Cn.rep = cluster_rep[ci];
        Cn.blk = P.blk;
        Cn.c0 = p;
        Cn.c1 = q;
        Cn.depth = P.depth + 1;
        Cn.dfok = dfok ? 1 : 0;
        Cn.dfexp = dfexp;
        Cn.sigma = P.sigma + tau;
        Cn.lnb = C.lnb - tau;
        Cn.rnb = C.rnb - tau;
        child_nodes[ci] = Cn;
        child_tau[ci] = tau;
        atomicAdd(&info->new_rrr, 1);
        if (untested) { atomicAdd(&info->untested, 1); atomicAdd(&info->status[MR3_SUNTESTED_RRR], 1); }
    }
}

__global__ void k_shift(int ncluster, const ClusterItem *__restrict__ clusters,
                        const long long *__restrict__ cluster_rep, const Node *__restrict__ nodes,
                        const BlkDesc *__restrict__ blks, const double *__restrict__ pool,
                        double *childpool, Node *child_nodes, double *child_tau, int *cnode,
                        int *active_list, const ShiftDecision *__restrict__ dec, int erep,
                        DevInfo *info, const int *dncluster) {
    // one warp per item; a grid smaller than the items loops over them
    const int nw_ = gridDim.x * (blockDim.x >> 5);
    const int bound_ = (dncluster ? *dncluster : ncluster);
    for (int ci = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ci < bound_; ci += nw_)
        k_shift_item(ci, ncluster, clusters, cluster_rep, nodes, blks, pool, childpool, child_nodes,
                     child_tau, cnode, active_list, dec, erep, info, dncluster);
}

size_t shift_scratch_bytes(int ncluster, int max_tries) {
    const size_t nc = (size_t)std::max(ncluster, 1);
    return nc * sizeof(ShiftDecision) + nc * (size_t)ladder_width(max_tries) * sizeof(double2) +
           (2 * nc + 2) * sizeof(int);
}

void launch_shift(int ncluster, const ClusterItem *clusters, const long long *cluster_rep,
                  const Node *nodes, const BlkDesc *blks, const double *pool, double *childpool,
                  Node *child_nodes, double *child_tau, int *cnode, int *active_list,
                  const int *jloc, double *lo, double *hi, int max_tries, unsigned fault_mask,
                  int erep, double2 *tri, void *ws, DevInfo *info, cudaStream_t s,
                  const int *dncluster) {
    (void)jloc;
    if (ncluster <= 0) return;
    // with a device count, ncluster is its bound: the grids and the scratch layout follow
    // the bound, the kernels the count
    const int NL = ladder_width(max_tries);
    ShiftDecision *dec = (ShiftDecision *)ws;
    double2 *lad = (double2 *)(dec + ncluster);
    int *ladder = (int *)(lad + (size_t)ncluster * NL);
    int *recomp = ladder + ncluster;
    int *counts = recomp + ncluster;
    cudaMemsetAsync(counts, 0, 2 * sizeof(int), s);
    // first candidates, one lane each (single-warp blocks keep the warps spread)
    k_shift_trials<<<(unsigned)((2ll * ncluster + 31) / 32), 32, 0, s>>>(
        ncluster, clusters, cluster_rep, nodes, blks, pool, childpool, lo, hi, fault_mask, tri,
        info, dncluster);
    const unsigned cb = (unsigned)((ncluster + 127) / 128);
    k_shift_select<<<cb, 128, 0, s>>>(ncluster, clusters, nodes, blks, lo, hi, fault_mask, tri,
                                      dec, ladder, counts, info, dncluster);
    // back-off ladder and the envelope test's backward recurrences of the queued clusters
    // (threads past the queue's length return), and the envelope test itself.  Few
    // clusters (latency bound): the ladder and the recurrences share one launch, and the
    // ladder's results for clusters the envelope test settles go unused.  Many clusters
    // (throughput bound): the envelope test first, and the ladder only for the rest.  The
    // decisions are the same either way.
    // with a device count the grids loop over the work (a few warps per SM each)
    const unsigned lfull = (unsigned)(((long long)ncluster * NL + 31) / 32);
    const unsigned efull = (unsigned)((2ll * ncluster + 31) / 32);
    const unsigned tfull = (unsigned)((ncluster + 3) / 4);
    const unsigned lblocks = dncluster ? std::min<unsigned>(lfull, 152 * 32) : lfull;
    const unsigned eblocks = dncluster ? std::min<unsigned>(efull, 152 * 32) : efull;
    const unsigned tblocks = dncluster ? std::min<unsigned>(tfull, 152 * 8) : tfull;
    // (with a device count both orders are launched, and the count picks one on the device)
    const bool few = ncluster < kEnvSequentialClusters;
    if (dncluster || few) {
        k_shift_ladder<<<lblocks + eblocks, 32, 0, s>>>(
            ncluster, max_tries, clusters, cluster_rep, nodes, blks, pool, childpool, lo, hi, tri,
            fault_mask, ladder, counts, dec, lad, lblocks, info, dncluster ? 1 : 0, dncluster);
    }
    if (dncluster || !few) {
        k_shift_ladder<<<eblocks, 32, 0, s>>>(
            ncluster, max_tries, clusters, cluster_rep, nodes, blks, pool, childpool, lo, hi, tri,
            fault_mask, ladder, counts, dec, lad, 0u, info, dncluster ? 2 : 0, dncluster);
    }
    k_shift_envtest<<<tblocks, 128, 0, s>>>(ncluster, clusters, cluster_rep, nodes, blks, pool,
                                            childpool, lo, hi, tri, fault_mask, ladder, counts,
                                            dec, info);
    if (dncluster || !few) {
        k_shift_ladder<<<lblocks, 32, 0, s>>>(
            ncluster, max_tries, clusters, cluster_rep, nodes, blks, pool, childpool, lo, hi, tri,
            fault_mask, ladder, counts, dec, lad, lblocks, info, dncluster ? 2 : 0, dncluster);
    }
    k_shift_pick<<<cb, 128, 0, s>>>(ncluster, max_tries, fault_mask, clusters, nodes, blks, lo, hi,
                                    tri, ladder, counts, lad, dec, recomp, info);
    k_shift_recompute<<<(unsigned)((ncluster + 31) / 32), 32, 0, s>>>(
        ncluster, clusters, cluster_rep, nodes, blks, pool, childpool, recomp, counts, dec, info);
    // conversion to the child representations, one warp per cluster
    k_shift<<<dncluster ? std::min(ncluster, 152 * 32) : ncluster, 32, 0, s>>>(
        ncluster, clusters, cluster_rep, nodes, blks, pool, childpool,
                                    child_nodes, child_tau, cnode, active_list, dec, erep, info,
                                    dncluster);
}

// ------------------------------------------------------------------ output order

// Per matrix (one warp): eigenvalues of a single block come out in order up to rounding
// (Rayleigh quotients of eigenvalues equal to working accuracy may differ by ulps in
// either direction): make them ascending by a running maximum, which moves a value by at
// most that rounding.  Matrices that split into several blocks come out block by block
// and are flagged for a sort.
__global__ void k_order_fix(int nmat, const MatDesc *__restrict__ mats, double *w, int *flags) {
    const int mi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (mi >= nmat) return;
    const MatDesc M = mats[mi];
    if (M.nblk > 1) {
        int bad = 0;
        for (int t = lane; t + 1 < M.m; t += 32) bad |= (w[M.woff + t] > w[M.woff + t + 1]);
        bad = __any_sync(FULL_MASK, bad);
        if (lane == 0) flags[mi] = bad;
        return;
    }
    double carry = -INFINITY;
    for (int base = 0; base < M.m; base += 32) {
        const int t = base + lane;
        double v = (t < M.m) ? w[M.woff + t] : -INFINITY;
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(FULL_MASK, v, o);
            if (lane >= o) v = fmax(v, y);
        }
        v = fmax(v, carry);
        if (t < M.m) w[M.woff + t] = v;
        carry = __shfl_sync(FULL_MASK, v, 31);
    }
    if (lane == 0) flags[mi] = 0;
}

void launch_order_flags(int nmat, const MatDesc *mats, double *w, int *flags, cudaStream_t s) {
    if (nmat > 0) k_order_fix<<<(nmat + 3) / 4, 128, 0, s>>>(nmat, mats, w, flags);
}

// Sort of one matrix's eigenpairs: the rank of each eigenvalue (ties by position) by one
// thread per eigenvalue over the values staged in shared-memory tiles, then a gather of
// the Z columns into a temporary and a copy back (one warp per column, coalesced).
__global__ void k_rank(const MatDesc *__restrict__ mats, int mi, const double *__restrict__ w,
                       int *perm, double *wtmp) {
    __shared__ double tile[1024];
    const MatDesc M = mats[mi];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const double x = (t < M.m) ? w[M.woff + t] : 0.0;
    int r = 0;
    for (int base = 0; base < M.m; base += 1024) {
        __syncthreads();
        for (int u = threadIdx.x; u < 1024; u += blockDim.x)
            tile[u] = (base + u < M.m) ? w[M.woff + base + u] : INFINITY;
        __syncthreads();
        const int lim = min(1024, M.m - base);
        for (int u = 0; u < lim; ++u) {
            const double y = tile[u];
            r += (y < x) || (y == x && base + u < t);
        }
    }
    if (t < M.m) {
        perm[t] = r;
        wtmp[r] = x;
    }
}

__global__ void k_gather_cols(const MatDesc *__restrict__ mats, int mi, const int *__restrict__ perm,
                              const double *__restrict__ Z, double *ztmp) {
    const MatDesc M = mats[mi];
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (col >= M.m) return;
    const double *src = Z + M.zoff + (long long)col * M.ldz;
    double *dst = ztmp + (long long)perm[col] * M.n;
    for (int i = lane; i < M.n; i += 32) dst[i] = src[i];
}

__global__ void k_copy_back(const MatDesc *__restrict__ mats, int mi, const double *__restrict__ wtmp,
                            const double *__restrict__ ztmp, double *w, double *Z) {
    const MatDesc M = mats[mi];
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (col >= M.m) return;
    if (lane == 0) w[M.woff + col] = wtmp[col];
    const double *src = ztmp + (long long)col * M.n;
    double *dst = Z + M.zoff + (long long)col * M.ldz;
    for (int i = lane; i < M.n; i += 32) dst[i] = src[i];
}

void launch_sort_outputs(int mi, int m, const MatDesc *mats, double *w, double *Z, double *wtmp,
                         double *ztmp, int *perm, cudaStream_t s) {
    if (m <= 1) return;
    k_rank<<<(m + 255) / 256, 256, 0, s>>>(mats, mi, w, perm, wtmp);
    k_gather_cols<<<(m + 7) / 8, 256, 0, s>>>(mats, mi, perm, Z, ztmp);
    k_copy_back<<<(m + 7) / 8, 256, 0, s>>>(mats, mi, wtmp, ztmp, w, Z);
}

cudaError_t preload_levels() {
    return load_kernels(k_bisect2, k_grid_counts, k_grid_bracket, k_classify, k_refine_ends,
                        k_shift_trials, k_shift_select, k_shift_envtest,
                        k_shift_ladder, k_shift_pick,
                        k_shift_recompute, k_shift, k_order_fix, k_rank, k_gather_cols,
                        k_copy_back);
}

} // namespace mr3
