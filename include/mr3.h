/*
 * mr3.h -- C ABI of the GB300 MRRR library (libmr3.so).
 *
 * The library computes eigenpairs (lambda_i, z_i) of a real symmetric tridiagonal
 * matrix T = tridiag(e, d, e) with the method of Multiple Relatively Robust
 * Representations (MRRR): the problem statement of the thesis' Alg. "MRRR"
 * (Sec. 3.1.2): input T by its diagonal and off-diagonal, an index set or value
 * interval; output eigenvalues and orthonormal eigenvectors.  The role matches
 * LAPACK's xSTEMR (App. A).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All floating-point data are IEEE binary64 (double).
 *  - "device" pointers are CUDA device (or managed) memory of the current device;
 *    "host" pointers are ordinary host memory (pinned memory is faster).
 *  - Matrices are column-major.  Z holds one eigenvector per column.
 *  - Eigenvalues are returned in ascending order; column j of Z belongs to w[j].
 *  - Each eigenvector has unit 2-norm and an entry of largest magnitude is positive
 *    (entries equal in magnitude in exact arithmetic are ordered by rounding).
 *  - The caller owns every array; the library never frees caller memory.  The
 *    library takes its internal workspace with stream-ordered allocation on the given
 *    stream from a memory pool of its own (see mr3_release_memory) and returns it to
 *    the pool before the call ends.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    All device work is enqueued on it.  The solver calls read a few counters back
 *    to the host (through a small mapped pinned buffer per host thread, allocated on
 *    first use, so that no copy engine is involved) and therefore synchronise with the
 *    stream before returning; the results are complete when the call returns.
 *  - Return value: 0 on success; -i when argument i (1-based) is invalid; a
 *    positive MR3_S* status when the result was produced but a safeguard fired
 *    (see mr3_info.status_counts); MR3_EOOM / MR3_ECUDA on resource errors.
 *  - Nothing here allocates or reads host memory passed as "device" or vice versa.
 */
#ifndef MR3_H
#define MR3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Which eigenpairs to compute (App. A / Sec. 3.2.1 remark 2). */
typedef enum {
    MR3_RANGE_ALL = 0,   /* all n eigenpairs                                  */
    MR3_RANGE_VALUE = 1, /* eigenvalues in the half-open interval (vl, vu]    */
    MR3_RANGE_INDEX = 2  /* eigenvalues il..iu (1-based, ascending)           */
} mr3_range;

/* Internal arithmetic of the representation tree (Ch. 5: FP64 in and out, the
 * tree either in FP64 or in double-double).  MR3_DD: representations, shifts
 * (dstqds), twisted factorizations and the Rayleigh-quotient iteration in
 * double-double (unit roundoff ~2^-104); eigenvalue approximation by bisection in
 * binary64 on the representations' leading words; gaptol 1e-10 by default; the RQI
 * stops at a local residual of gap * eps * sqrt(n).  Expected orthogonality
 * ~eps sqrt(n) instead of the FP64 tree's O(n eps / gaptol) worst case. */
typedef enum { MR3_FP64 = 0, MR3_DD = 1 } mr3_precision;

/* Options; a zero-initialised struct (or NULL) selects the defaults in brackets. */
typedef struct {
    int prec;                  /* mr3_precision [MR3_FP64]                                   */
    double gaptol;             /* classification threshold on reldist (Sec. 3.2.3)
                                  [FP64: max(1e-3, min(2/n_b, 0.05)) for an irreducible
                                  block of order n_b, so that the tree's loss of
                                  orthogonality, ~eps/gaptol, stays below 10 n eps at small
                                  n; DD: 1e-10 (Ch. 5, Eq. gaptolinterval)]               */
    unsigned long long seed;   /* stream of the root's random perturbation (Alg. MRRR)
                                  [0x5EED]                                                   */
    int max_rqi;               /* Rayleigh-quotient iterations per singleton before the
                                  bisection fallback (Alg. S-task) [10]                      */
    int max_shift_tries;       /* back-off steps per side when shifting a cluster
                                  (Alg. "Shifting the spectrum") [8]                        */
    unsigned fault_mask;       /* MR3_FAULT_* bits: host-selected fault injection [0]        */
    int tpe;                   /* bisection lanes per eigenvalue: 0 = auto, else 1..32       */
    int max_depth;             /* cap on the representation-tree depth [64]                  */
    int profile;               /* nonzero: time each kernel group with CUDA events on the
                                  call's stream and report it in mr3_info.kernel_ms [0].
                                  Diagnostics: with MR3_TRACE=1 in the environment the
                                  host-driven level loop also prints one line per tree level
                                  on stderr (counts, main-stream times of the level's cluster
                                  ends, shifts and child bisection, and the sweep statistics
                                  of its multisection launches); it synchronises the stream
                                  once per level                                             */
    int rqi_team;              /* lanes per singleton in the RQI: 0 = auto (2 for many
                                  singletons, else 8), 2 or 8 to force one; mr3_stemr_static
                                  always uses 8 [0]                                          */
    int bisect_warps;          /* bisection lanes per eigenvalue are chosen to keep about this
                                  many warps per SM in flight: 0 = 48, else 1..64 (tpe > 0
                                  overrides) [0]                                              */
    int abs_split;             /* the root's classification also separates neighbours whose
                                  absolute gap is at least the block's average gap
                                  spdiam / (n_b - 1) (the relative criterion amended by
                                  absolute gaps, Sec. 3.2.3, Sec. 4.2.1); the pieces cut out
                                  of a relative cluster get their own representations.
                                  Positive = on.  Caution: those representations are shifted
                                  into the interior of the root's spectrum, where element
                                  growth can fail the growth test on every candidate (near-
                                  Toeplitz spectra); they are then accepted by least growth,
                                  the call returns MR3_SUNTESTED_RRR, and orthogonality is
                                  no longer guaranteed.  mr3_stemr_static never applies it
                                  [0: relative gaps only]                                    */
    int erep;                  /* nonzero: binary64 child representations are kept as
                                  e-representations (d, beta): the off-diagonal entries are
                                  shared with the root instead of recomputed as d+ l+ (Ch. 3,
                                  representation forms; Ch. 5).  The double-double tree always
                                  works this way [0]                                         */
    int graph;                 /* the tree's level loop captured in one CUDA graph (no host
                                  read-back between levels): 0 = for solves of 2 or more
                                  matrices unless profile is set, 1 = always, -1 = never.  Binary64 tree only,
                                  without abs_split; a tree deeper than the graph's 12
                                  levels, or representations that overflow its fixed arenas,
                                  are redone by the host-driven loop (same results) [0]      */
} mr3_opts;

/* Fault injection (tests of the safeguards; nothing here faults a GPU). */
#define MR3_FAULT_RQI_NOCONV   0x1u /* RQI never accepts: forces the bisection fallback   */
#define MR3_FAULT_SHIFT_REJECT 0x2u /* every shifted representation fails the growth test */
#define MR3_FAULT_NAN_SHIFT    0x4u /* the first shift candidate of each cluster is NaN   */

/* Algorithmic status codes (positive return values) and their counters. */
#define MR3_SOK             0
#define MR3_SUNTESTED_RRR   1 /* a cluster representation was accepted untested (least growth) */
#define MR3_SCAP            2 /* an iteration cap was hit for some eigenpair              */
#define MR3_SNONFINITE      3 /* non-finite input                                         */
#define MR3_SDEPTH          4 /* the tree depth cap was reached                           */
#define MR3_EOOM            5 /* out of device memory                                     */
#define MR3_ECUDA           6 /* a CUDA call failed                                       */
#define MR3_ENOSCRATCH      7 /* request exceeds a fixed-size internal buffer             */

/* Statistics of one call (Sec. 2.5 and Ch. 5 measures). */
typedef struct {
    int m;                     /* eigenpairs computed                                     */
    int nblocks;               /* irreducible blocks after splitting (Sec. 3.2.1)         */
    int dmax;                  /* depth of the representation tree (Sec. 3.1.2)           */
    int nclusters;             /* cluster nodes processed                                 */
    int largest_cluster;       /* size of the largest cluster (clustering rho * n, Ch. 5) */
    int new_rrr;               /* representations computed for clusters                   */
    int untested_rrr;          /* of those, accepted by least growth only (phi, Ch. 5)    */
    long long rqi_iters;       /* Rayleigh-quotient iterations, summed                    */
    int rqi_iters_max;         /* ... maximum over eigenpairs                             */
    int bisect_fallbacks;      /* singletons finished by bisection + one Getvec           */
    long long sturm_steps;     /* Sturm-count steps of the bisection kernel (work measure) */
    long long shift_steps;     /* recurrence steps of the cluster-shift kernel              */
    long long twisted_steps;   /* recurrence steps inside the singleton (RQI) kernel        */
    int status_counts[8];      /* occurrences of each MR3_S* code                          */
    /* With opts->profile: device time (ms) and launches per kernel group, measured with
       CUDA events on the call's stream.  Groups: 0 prologue (norms, splitting, ranges),
       1 root representation, 2 bisection on the root, 3 classification, 4 singletons (RQI),
       5 cluster shifts, 6 refinement on child representations, 7 output ordering. */
    double kernel_ms[8];
    int kernel_launches[8];
    int ladder_clusters;       /* clusters whose first two shift candidates (tau_l, tau_r at
                                  the refined ends) both failed the plain growth test       */
    int recomputed_rrr;        /* ... of those, clusters a back-off candidate then passed  */
    int envelope_rrr;          /* ... of those, clusters a first candidate of which passed
                                  the envelope-weighted growth test (Alg. "Shifting the
                                  spectrum", remark 3)                                      */
    int graph_levels;          /* levels run inside the graph-captured loop (0: host loop);
                                  with it, kernel_ms[3] holds the levels' time and groups
                                  4-6 stay 0                                                */
    int graph_runs;            /* graph launches (2 after an arena overflow)                */
    long long graph_pool_peak; /* largest arena need (doubles) of the last graph launch     */
} mr3_info;

/*
 * mr3_stemr -- selected eigenpairs of one symmetric tridiagonal matrix.
 *
 *  n      (1)  order of T, n >= 0.
 *  d      (2)  device, n doubles: diagonal alpha_1..alpha_n.
 *  e      (3)  device, n-1 doubles: off-diagonal beta_1..beta_{n-1} (may be NULL if n <= 1).
 *  range  (4)  mr3_range.
 *  vl, vu (5,6) MR3_RANGE_VALUE: interval (vl, vu], vl < vu.  Ignored otherwise.
 *  il, iu (7,8) MR3_RANGE_INDEX: 1 <= il <= iu <= n (or il = 1, iu = 0 when n = 0).
 *  m      (9)  host int, out: number of eigenpairs found.
 *  w      (10) device, out: m ascending eigenvalues (room for n when range = VALUE).
 *  Z      (11) device, out: n x m column-major, leading dimension ldz.
 *  ldz    (12) ldz >= max(1, n).
 *  opts   (13) host, may be NULL.
 *  info   (14) host, out, may be NULL.
 *  stream (15) cudaStream_t as void*.
 * Splitting (Sec. 3.2.1): off-diagonals with |beta_i| <= eps sqrt(n) ||T|| are
 * treated as zero and each block is solved on its own; rows of a column outside
 * its block are zero.
 */
int mr3_stemr(int n, const double *d, const double *e, int range, double vl, double vu,
              int il, int iu, int *m, double *w, double *Z, int ldz,
              const mr3_opts *opts, mr3_info *info, void *stream);

/*
 * mr3_stemr_host -- mr3_stemr on host arrays: the library copies d and e to the
 * device, solves, and copies w (m values) and Z (n x m, leading dimension ldz) back
 * into the caller's host arrays before returning.  Arguments as for mr3_stemr with
 * host pointers.
 */
int mr3_stemr_host(int n, const double *d, const double *e, int range, double vl, double vu,
                   int il, int iu, int *m, double *w, double *Z, int ldz,
                   const mr3_opts *opts, mr3_info *info, void *stream);

/*
 * mr3_stemr_batched -- eigenpairs of nb independent tridiagonals of uneven sizes.
 *
 *  nb     (1)  number of matrices, nb >= 0.
 *  n_off  (2)  host, nb+1 int64: matrix b has order n_b = n_off[b+1]-n_off[b] >= 0 and
 *              occupies d[n_off[b] .. n_off[b+1]) and e[n_off[b] .. n_off[b+1]-1).
 *  d      (3)  device, n_off[nb] doubles (packed diagonals).
 *  e      (4)  device, n_off[nb] doubles (packed off-diagonals; the last slot of
 *              each matrix is not read).
 *  range  (5)  mr3_range, the same for every matrix.
 *  vl, vu (6,7) host, nb doubles each (range VALUE), else may be NULL.
 *  il, iu (8,9) host, nb ints each (range INDEX), else may be NULL.
 *  m      (10) host, out, nb ints: eigenpairs found per matrix.
 *  w      (11) device, out: eigenvalues of matrix b at w[n_off[b] ..] (room for n_b).
 *  z_off  (12) host, nb int64: Z_b starts at Z + z_off[b] and is n_b x n_b
 *              column-major with leading dimension n_b (room for n_b columns).
 *  Z      (13) device, out.
 *  opts   (14), info (15) as for mr3_stemr (info sums over the batch), stream (16).
 */
int mr3_stemr_batched(int nb, const long long *n_off, const double *d, const double *e,
                      int range, const double *vl, const double *vu, const int *il,
                      const int *iu, int *m, double *w, const long long *z_off, double *Z,
                      const mr3_opts *opts, mr3_info *info, void *stream);

/*
 * mr3_stemr_batched_host -- mr3_stemr_batched on host arrays: the library copies d and e
 * (n_off[nb] doubles each, packed as for mr3_stemr_batched) to the device, solves, and
 * copies each matrix's m[b] eigenvalues to w[n_off[b] ..] and its n_b x m[b] eigenvectors
 * to Z + z_off[b] (leading dimension n_b) in the caller's host arrays before returning.
 * Arguments as for mr3_stemr_batched with host pointers for d, e, w and Z (pinned host
 * memory is copied fastest); the device workspace, outputs included, comes from the
 * library's pool and is returned to it.  Entries of w and Z beyond m[b] are not written.
 */
int mr3_stemr_batched_host(int nb, const long long *n_off, const double *d, const double *e,
                           int range, const double *vl, const double *vu, const int *il,
                           const int *iu, int *m, double *w, const long long *z_off, double *Z,
                           const mr3_opts *opts, mr3_info *info, void *stream);

/*
 * mr3_backward -- gradient of a scalar loss L(lambda, Z) with respect to d and e,
 * given the forward eigen-decomposition of T (all n eigenpairs) and the upstream
 * gradients g = dL/dlambda and G = dL/dZ.
 *
 *   dbar_j = sum_i g_i z_ij^2 + Abar_jj,   ebar_j = 2 sum_i g_i z_ij z_i,j+1 + Abar_j,j+1 + Abar_j+1,j
 *   Abar   = Z (F o (Z^T G)) Z^T  with  F_ik = 1/(lambda_k - lambda_i) (i != k), F_ii = 0,
 *            regularised as (lambda_k - lambda_i)/((lambda_k - lambda_i)^2 + delta^2),
 *            delta = n eps ||T|| (pairs closer than the solver can resolve).
 *
 *  n      (1)  order, n >= 0;  k (2) number of eigenpairs in w/Z: must equal n when G
 *              is given; any 0 <= k <= n when G is NULL (eigenvalue part only).
 *  w      (3)  device, k eigenvalues (ascending).
 *  Z      (4)  device, n x k, leading dimension ldz (5) >= max(1, n).
 *  gw     (6)  device, k doubles, or NULL (treated as 0).
 *  gZ     (7)  device, n x k, leading dimension ldgz (8), or NULL (treated as 0).
 *  dd     (9)  device, out, n doubles;  de (10) device, out, n-1 doubles.
 *  opts   (11) may be NULL;  stream (12).
 */
int mr3_backward(int n, int k, const double *w, const double *Z, int ldz, const double *gw,
                 const double *gZ, int ldgz, double *dd, double *de, const mr3_opts *opts,
                 void *stream);

/*
 * mr3_backward_solve -- the gradient of mr3_backward for any number k of eigenpairs (a
 * subset included), with the eigenvector part computed one eigenpair at a time in O(n)
 * work each instead of by two dense n x n x n products.  Since dz_k = -(T - lambda_k I)^+
 * dT z_k, the eigenvector part of Tbar is -sum_k w_k z_k^T with w_k = (T - lambda_k I)^+ G_k,
 * solved by tridiagonal Gaussian elimination with partial pivoting and projected off z_k
 * (backward stable: the near-singular direction carries only rounding).  Eigenvalues
 * closer than 1e-6 ||T|| to each
 * other (up to 64 in a row) form a group: their components are projected out of the solve
 * and their pairs use the regularised dense formula of mr3_backward.  With a subset, the
 * result is exact for a loss of the computed eigenpairs as long as no eigenvalue outside
 * the computed range lies within 1e-6 ||T|| of a computed one.
 *
 *  n (1), k (2) 0 <= k <= n;  d (3), e (4) device: T's diagonal (n) and off-diagonal (n-1);
 *  w (5) device, k ascending eigenvalues;  Z (6) device n x k, ldz (7) >= max(1, n);
 *  gw (8) device k doubles or NULL;  gZ (9) device n x k or NULL, ldgz (10);
 *  dd (11) device out n;  de (12) device out n-1;  opts (13) may be NULL;  stream (14).
 *  Device workspace: 4 n k + O(n) doubles from the library's pool.  Synchronises the
 *  stream before returning.  Returns 0, -i for an invalid argument i, MR3_EOOM, MR3_ECUDA.
 */
int mr3_backward_solve(int n, int k, const double *d, const double *e, const double *w,
                       const double *Z, int ldz, const double *gw, const double *gZ, int ldgz,
                       double *dd, double *de, const mr3_opts *opts, void *stream);

/*
 * mr3_stemr_static -- mr3_stemr for one matrix of order n <= MR3_STATIC_MAX_N, with all
 * device workspace inside a fixed array of MR3_STATIC_SCRATCH_BYTES that the library
 * holds on each device: the call allocates no device memory.  The thesis has no
 * counterpart; this entry point exists for callers that cannot let a library allocate
 * (their device memory is claimed in full up front, or no allocator may be entered).
 *
 *  Arguments, outputs, defaults and return codes as for mr3_stemr, except that
 *  opts->prec must be MR3_FP64 (else -13) and opts->profile is ignored (kernel_ms and
 *  kernel_launches stay zero).  Every step runs on `stream`.
 *  Extra return code: MR3_ENOSCRATCH when n > MR3_STATIC_MAX_N (checked before any
 *  device work), or when the representation tree of this matrix needs more room than
 *  the array has (then w and Z are undefined, *m = 0, and the stream is idle on return).
 *  Set-up: the first call made with a device current and n <= MR3_STATIC_MAX_N (n = 0
 *  is enough) loads, on that device, every kernel this entry point launches and the
 *  array itself (the runtime would otherwise load each kernel at its first launch, which
 *  takes device memory), and looks up and caches the array's address.  A caller that
 *  claims its device memory up front makes that first call before claiming it; the first
 *  call on each device should also come before any stream capture begins.
 *  Sharing: one array per device.  Calls that overlap in time on the same device (other
 *  host threads, or streams not ordered with respect to each other) race on it: order them.
 */
#define MR3_STATIC_SCRATCH_BYTES (32u << 20) /* 32 MiB per device                 */
#define MR3_STATIC_MAX_N 1024                /* largest order mr3_stemr_static takes */
int mr3_stemr_static(int n, const double *d, const double *e, int range, double vl, double vu,
                     int il, int iu, int *m, double *w, double *Z, int ldz,
                     const mr3_opts *opts, mr3_info *info, void *stream);

/* Device memory.  The workspaces of mr3_stemr, mr3_stemr_host, mr3_stemr_batched and
 * mr3_backward come from a stream-ordered memory pool that the library keeps per device,
 * created on the first call made with that device current.  Memory a call frees stays in
 * the pool for the next call instead of going back to the driver at each synchronisation
 * (re-mapping several GB per call costs tens of ms).  mr3_release_memory returns the
 * unused memory of every pool to the driver; memory still held by calls in flight stays.
 * Thread-safe; returns MR3_SOK, or MR3_ECUDA if a CUDA call failed. */
int mr3_release_memory(void);

/* Message for a return code (static string). */
const char *mr3_strerror(int code);

/* Library version string, e.g. "mr3-gb300 0.1 sm_103a". */
const char *mr3_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MR3_H */
