/*
 * gtb.h -- C ABI of libgtb, B300-native (sm_103a) stencils for weather and
 * climate codes: the horizontal-diffusion (hdiff) and vertical-advection
 * (vadv) benchmark stencils of the GT4Py paper (arXiv 2311.08322, Sec. 3.1),
 * their adjoints, and batched ensembles of uneven domains.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Fields are storages with halos (the paper's `storage`, Sec. 2.2/2.3): a
 * gtb_field describes caller-owned DEVICE memory.  Element (i,j,k) of the
 * storage is at  ptr + i*strides[0] + j*strides[1] + k*strides[2]  (strides in
 * elements; strides[0] must be 1, i.e. i is the contiguous axis, and the
 * layout must be non-overlapping: strides[1] >= shape[0],
 * strides[2] >= strides[1]*shape[1]).  `origin` is the storage index of compute
 * domain point (0,0,0) of that field, exactly as the paper's `origin` call
 * argument (Sec. 2.2).  `domain` (I,J,K) is the compute domain; pass NULL to
 * have it deduced from the field sizes and the stencil's reach (Sec. 2.2: the
 * iteration space is deduced from field sizes and stencil shape): the largest
 * domain for which every access of every field stays inside its storage.
 *
 * Every field of one call has the same dtype (GTB_F32 or GTB_F64).
 *
 * Ownership: the library never allocates, frees or retains caller memory, and
 * never synchronises: each call validates its arguments on the host, enqueues
 * its kernels on `stream` (a cudaStream_t; NULL = the legacy default stream)
 * and returns.  An empty domain (any extent 0) enqueues nothing and succeeds.
 *
 * Errors: every call returns GTB_OK (0) or a negative gtb_status; on error
 * nothing is enqueued and gtb_last_error() returns a message for the calling
 * thread.  Argument checks are the paper's run-time checks on storage layout
 * and data type (Sec. 3.1), done in C at a cost of well under a microsecond.
 * Kernels never trap: a device-side wait that runs out of its time limit
 * records GTB_ERR_DEVICE, which gtb_device_status() reports.
 *
 * Checked build: libgtb_checked.so exports the same entry points with the same
 * results; before its first access each kernel tests the ends of every run of
 * addresses it will touch against the storage its gtb_field declares (shape and
 * strides from ptr), and a run outside it is not accessed and records
 * GTB_ERR_DEVICE as well (the library's own index arithmetic under test, in
 * place of a memory sanitizer).  Slower; for debugging and tests.
 */
#ifndef GTB_H
#define GTB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GTB_OK = 0,
    GTB_ERR_NULL = -1,        /* a required pointer is NULL */
    GTB_ERR_DTYPE = -2,       /* unknown dtype, or fields of one call differ */
    GTB_ERR_EXTENT = -3,      /* origin/domain plus stencil reach leaves a storage */
    GTB_ERR_LAYOUT = -4,      /* strides[0] != 1, negative or overlapping strides */
    GTB_ERR_ALIAS = -5,       /* an output overlaps an input it may not overlap */
    GTB_ERR_LAUNCH = -6,      /* the CUDA launch failed (see gtb_last_error) */
    GTB_ERR_DEVICE = -7,      /* a kernel's bounded wait expired (device status) */
    GTB_ERR_UNSUPPORTED = -8, /* size beyond a documented limit */
    GTB_ERR_ARG = -9          /* bad scalar argument (prec, flags, counts) */
} gtb_status;

typedef enum { GTB_F32 = 1, GTB_F64 = 2 } gtb_dtype;

typedef struct gtb_field {
    void *ptr;           /* device address of storage element (0,0,0) */
    int32_t dtype;       /* gtb_dtype */
    int32_t reserved;    /* must be 0 */
    int64_t shape[3];    /* storage extents (ni, nj, nk) */
    int64_t strides[3];  /* element strides (1, sj, sk) */
    int64_t origin[3];   /* storage index of compute-domain point (0,0,0) */
} gtb_field;

/* Precision of the vadv column arithmetic (coefficients, right-hand side,
 * Thomas recurrences, output).  Storage precision is the fields' dtype. */
typedef enum {
    GTB_PREC_NATIVE = 0, /* arithmetic in the storage type */
    GTB_PREC_F64 = 1,    /* binary64 arithmetic on the FP64 pipe (F32 storage) */
    GTB_PREC_DF = 2      /* double-float (pairs of binary32, ~48-bit) on the FP32 pipe */
} gtb_prec;

/* flags */
#define GTB_WCON_LITERAL 1u   /* vadv: use wcon(i) as the face velocity instead of the I-face average */
#define GTB_ADJ_ACCUMULATE 2u /* adjoints: add into the cotangent outputs instead of overwriting them */
#define GTB_SAVE_FACTORS 4u   /* gtb_hdiff_vadv: keep the column factors (c'_k, 1/p_k) in the workspace */
#define GTB_ADJ_FACTORS 8u    /* gtb_vadv_adj: the workspace holds those factors; use them, do not refactorise */
#define GTB_STATE48 16u       /* gtb_vadv, GTB_F32 + GTB_PREC_DF: column state in the workspace in 48 bits */

/*
 * gtb_hdiff -- horizontal diffusion (paper Sec. 3.1; one PARALLEL computation,
 * Sec. 2.2, whose temporaries lap/fx/fy never reach memory, Sec. 2.2):
 *   lap = 4 in - (((in[i+1] + in[i-1]) + in[j+1]) + in[j-1])     on the domain and a 1-ring
 *   fx  = lap[i+1] - lap[i], set to 0 where fx * (in[i+1] - in[i]) > 0;  fy likewise in j
 *   out = in - coeff * ((fx[i] - fx[i-1]) + (fy[j] - fy[j-1]))
 * in:    read on the domain plus a 2-point ring in I and J (origin >= 2 there).
 * coeff: read on the domain.  out: written on the domain only.
 * out must not overlap in or coeff (GTB_ERR_ALIAS): in a PARALLEL stencil with
 * offsets the result may not overwrite its own input (Sec. 2.2).
 * FP64 results agree with a binary64 reference within 1e-12 (max-norm
 * relative); FP32 computes in binary32.
 */
int gtb_hdiff(const gtb_field *in, const gtb_field *coeff, const gtb_field *out,
              const int64_t *domain, void *stream);

/*
 * gtb_vadv -- implicit vertical advection (paper Sec. 3.1: vertically
 * sequential stages implementing a tridiagonal solver; a FORWARD computation
 * followed by a BACKWARD one with specialised top and bottom intervals, Sec. 2.2).
 * Per (i,j) column of K levels, with w_k = (wcon[i,k] + wcon[i+1,k]) / 2
 * (or wcon[i,k] with GTB_WCON_LITERAL), bp = (1+beta_v)/2, bm = (1-beta_v)/2:
 *   a_k  = bp (-w_k/2),  as_k = bm (-w_k/2)        (a_0 = as_0 = 0)
 *   c_k  = bp (w_{k+1}/2), cs_k = bm (w_{k+1}/2)   (c_{K-1} = cs_{K-1} = 0)
 *   b_k  = dtr_stage - a_k - c_k,
 *   d_k  = dtr_stage u_pos + utens + utens_stage
 *          - as_k (u_stage[k-1] - u_stage[k]) - cs_k (u_stage[k+1] - u_stage[k])
 *   solve A x = d by Thomas elimination (forward sweep, then back substitution),
 *   utens_stage_out = dtr_stage (x - u_pos).
 * At beta_v = 0: a_k = -w_k/4, c_k = w_{k+1}/4 (the benchmark coefficients).
 * wcon is read at i and i+1 (staggered in I; needs one halo point above I).
 * utens_stage_out may be the very same view as utens_stage (in place: each
 * column is read completely before it is written); any other overlap of the
 * output with an input is GTB_ERR_ALIAS.
 * prec: gtb_prec.  For GTB_F64 storage only GTB_PREC_NATIVE is accepted
 * (binary64); for GTB_F32 storage NATIVE is all-binary32, F64 and DF keep the
 * whole column computation in binary64 / double-float.
 * flags: GTB_WCON_LITERAL; GTB_STATE48 (GTB_F32 storage with GTB_PREC_DF only,
 * else GTB_ERR_ARG): the forward sweep stores c'_k and the back-substitution
 * term in the workspace as their binary32 high part and the top 16 bits of
 * their low part (12 bytes per point instead of 16, less DRAM traffic when the
 * column state outgrows L2); the back substitution then starts from values
 * within 2^-32 of the computed ones.  The max-norm error stays that of the
 * full-width form, but a column whose outputs are small beside its intermediate
 * values loses accuracy (worst column 9e-4 relative at 512x512x80, against
 * 6e-8).  Without a workspace the flag has no effect (shared-memory state).
 * A zero pivot (singular leading minor) yields non-finite values in that column,
 * as the unpivoted method does.  Limit without a workspace: K <= 448 (the column
 * state then lives in shared memory); larger K is GTB_ERR_UNSUPPORTED unless a
 * workspace of gtb_vadv_workspace_bytes() bytes is passed.
 *
 * workspace: optional caller-owned device scratch for the forward sweep's
 * column state (c'_k, and s_k = u_stage_k + u_pos_k or a back-substitution term),
 * at least gtb_vadv_workspace_bytes() bytes, 16-byte aligned, overlapping no
 * field; its contents on entry are ignored and on exit unspecified, and two
 * calls that may run concurrently need distinct workspaces.  With it the
 * kernel keeps no per-column state in shared memory and runs at full
 * occupancy (the fast form on B300, whose FP64 pipe needs many resident warps);
 * with NULL (or too small) the state stays in shared memory.
 */
int gtb_vadv(const gtb_field *u_stage, const gtb_field *wcon, const gtb_field *u_pos,
             const gtb_field *utens, const gtb_field *utens_stage,
             const gtb_field *utens_stage_out, double dtr_stage, double beta_v,
             int prec, unsigned flags, const int64_t *domain,
             void *workspace, size_t workspace_bytes, void *stream);

/* Bytes of workspace gtb_vadv uses for this dtype, prec and domain (I,J,K):
 * K*I*J*16 for GTB_F64 storage, K*I*J*4 for GTB_F32 with GTB_PREC_NATIVE,
 * K*I*J*16 for GTB_F32 with GTB_PREC_F64 or GTB_PREC_DF; 0 for bad arguments. */
size_t gtb_vadv_workspace_bytes(int dtype, int prec, const int64_t *domain);

/*
 * gtb_hdiff_adj -- reverse mode of gtb_hdiff (the differentiation form of the
 * paper's horizontal-diffusion benchmark, Sec. 3.1): a transposed stencil
 * whose limiter keep/zero decisions are recomputed from `in` (the map is
 * linear on each piece of the limiter).  Given out_bar on the domain:
 *   in_bar    = out_bar - (dD/din)^T (coeff * out_bar)   written on the domain
 *               plus its 2-point ring in I and J (overwritten; needs origin >= 2)
 *   coeff_bar = -D * out_bar on the domain (optional, NULL to skip; added to
 *               the existing values with GTB_ADJ_ACCUMULATE, else overwritten)
 * D is the forward flux divergence.  in_bar and coeff_bar may not overlap any
 * input or each other (GTB_ERR_ALIAS).  Limit: K <= 65535.
 */
int gtb_hdiff_adj(const gtb_field *in, const gtb_field *coeff, const gtb_field *out_bar,
                  const gtb_field *in_bar, const gtb_field *coeff_bar, unsigned flags,
                  const int64_t *domain, void *stream);

/*
 * gtb_vadv_adj -- reverse mode of gtb_vadv for fixed wcon (the transposed
 * tridiagonal solve of the paper's implicit vertical solver, Sec. 3.1, run as
 * a forward sweep with U^T and a backward sweep with L^T of A = LU).  The
 * output utens_stage_out is linear in (u_stage, u_pos, utens, utens_stage):
 *   z = A^-T (dtr_stage * y_bar),
 *   utens_bar = utens_stage_bar = z,  u_pos_bar = dtr_stage (z - y_bar),
 *   u_stage_bar = E^T z  (E: the explicit correction of the right-hand side).
 * Every output is optional (NULL); outputs are overwritten, or added to with
 * GTB_ADJ_ACCUMULATE.  u_stage_bar and u_pos_bar may be the very same view:
 * it then receives their sum (the cotangent of a field passed as both
 * u_stage and u_pos).  No other output may overlap an input or another output.
 * flags: GTB_WCON_LITERAL, GTB_ADJ_ACCUMULATE, GTB_ADJ_FACTORS.  workspace: as
 * for gtb_vadv, of gtb_vadv_adj_workspace_bytes() bytes.  With GTB_ADJ_FACTORS
 * the workspace is REQUIRED and must hold the factors that gtb_hdiff_vadv kept
 * with GTB_SAVE_FACTORS for the same wcon, dtr_stage, beta_v, prec, flags
 * and domain (c'_k, then 1/p_k); the forward sweep then reads them instead of
 * refactorising A (the same values, so the same results), and overwrites
 * them: each set of factors serves one adjoint.  Limit without a workspace:
 * K <= 448 (GTB_ERR_UNSUPPORTED beyond).
 */
int gtb_vadv_adj(const gtb_field *wcon, const gtb_field *y_bar, const gtb_field *u_stage_bar,
                 const gtb_field *u_pos_bar, const gtb_field *utens_bar, const gtb_field *utens_stage_bar,
                 double dtr_stage, double beta_v, int prec, unsigned flags, const int64_t *domain,
                 void *workspace, size_t workspace_bytes, void *stream);

/* Workspace bytes of gtb_vadv_adj: 2*K*I*J times 8 (GTB_F64, or GTB_F32 with
 * GTB_PREC_F64 / GTB_PREC_DF) or 4 (GTB_F32, GTB_PREC_NATIVE). */
size_t gtb_vadv_adj_workspace_bytes(int dtype, int prec, const int64_t *domain);

/*
 * gtb_halo_periodic -- fill the hi-wide I halo and hj-wide J halo around the
 * domain with the periodic continuation of the domain (corners included), the
 * boundary condition of chained steps.  hi <= I and hj <= J.
 * gtb_halo_periodic_adj -- its adjoint: every domain point adds the values
 * held by the halo points that copy it; the halo itself is left unchanged.
 */
int gtb_halo_periodic(const gtb_field *f, int hi, int hj, const int64_t *domain, void *stream);
int gtb_halo_periodic_adj(const gtb_field *f, int hi, int hj, const int64_t *domain, void *stream);

/*
 * gtb_hdiff_vadv -- the two stencils chained as one computation (paper
 * Sec. 3.1; Sec. 2.2 leaves the backend free to fuse the computations it
 * runs):
 *   h               = hdiff(in, coeff)                          (as gtb_hdiff)
 *   utens_stage_out = vadv(u_stage = h, wcon, u_pos = h, utens, utens_stage)
 * GTB_F64 storage: in one kernel; h is formed level by level on chip and never
 * written to memory.  The back substitution runs on z = x - h (the same
 * unknowns, utens_stage_out = dtr_stage z), and h's update may be formed in
 * fixed point as in gtb_step, so results agree with gtb_hdiff followed by
 * gtb_vadv to rounding, not bit for bit.  GTB_F32 storage: the two kernels of
 * gtb_hdiff and gtb_vadv back to back on the stream, h in the workspace (on
 * B300 the HBM-bound binary32 hdiff and the FP32-pipe column solve run faster
 * apart than sharing SMs), with gtb_vadv's results bit for bit.
 * Fields: in needs 2 halo points in I and J (as gtb_hdiff), wcon one point
 * above I unless GTB_WCON_LITERAL (as gtb_vadv); coeff, utens, utens_stage
 * and utens_stage_out cover the domain.  utens_stage_out may be the very same
 * view as utens_stage (in place); any other overlap of the output with an
 * input is GTB_ERR_ALIAS.  dtr_stage, beta_v and prec as gtb_vadv.
 * workspace: REQUIRED caller-owned device scratch of at least
 * gtb_hdiff_vadv_workspace_bytes() bytes (c', e when it cannot be parked in
 * the output, and h for GTB_F32 storage), 16-byte aligned, overlapping no
 * field; NULL or too small is GTB_ERR_ARG.  No K limit beyond the workspace
 * size.
 * flags: GTB_WCON_LITERAL, GTB_SAVE_FACTORS (any other flag, GTB_STATE48
 * included, is GTB_ERR_ARG: the chained call keeps its column state at full
 * width).  With GTB_SAVE_FACTORS the
 * workspace keeps, on return, the factors of the column solve for the adjoint
 * (gtb_vadv_adj with GTB_ADJ_FACTORS): c'_k in its first K*I*J values and
 * 1/p_k in the next K*I*J (value type: binary64, or binary32 / binary64 /
 * double-float pairs as prec selects for GTB_F32 storage; index
 * k*I*J + j*I + i).
 */
int gtb_hdiff_vadv(const gtb_field *in, const gtb_field *coeff, const gtb_field *wcon,
                   const gtb_field *utens, const gtb_field *utens_stage,
                   const gtb_field *utens_stage_out, double dtr_stage, double beta_v,
                   int prec, unsigned flags, const int64_t *domain,
                   void *workspace, size_t workspace_bytes, void *stream);

/* Workspace bytes of gtb_hdiff_vadv for this dtype, prec, flags (with or
 * without GTB_SAVE_FACTORS) and domain; 0 for bad arguments. */
size_t gtb_hdiff_vadv_workspace_bytes(int dtype, int prec, unsigned flags, const int64_t *domain);

/*
 * gtb_step -- one step of the paper's benchmark (Sec. 3.1): both stencils on
 * their own fields,
 *   hdiff_out       = hdiff(in, coeff)                                (as gtb_hdiff)
 *   utens_stage_out = vadv(u_stage, wcon, u_pos, utens, utens_stage)  (as gtb_vadv)
 * For GTB_F64 storage the two are co-scheduled in one kernel: every CTA runs
 * the hdiff of a 32 x 2 column tile on two warps and the vadv column solve of
 * the same tile on two others (binary64 hdiff runs on the integer pipe and the
 * solve on the FP64 pipe, so the two overlap in every SM); hdiff_out then
 * equals gtb_hdiff's to rounding (the fixed-point scale is chosen per tile and
 * level, not per strip; and when the grid fills the GPU the update
 * in - coeff D is formed in that fixed point too, on the integer pipe, within
 * 2^-54 of the level's largest input).  For GTB_F32 storage (HBM-bound hdiff, FP32-pipe
 * solve) the two kernels run back to back, which is faster there, and
 * hdiff_out equals gtb_hdiff's.  utens_stage_out always equals gtb_vadv's
 * result (workspace form) bit for bit.
 * Both stencils share one domain (deduced from all nine fields when NULL).
 * Reach and in-place rules: as gtb_hdiff and gtb_vadv; hdiff_out may overlap
 * no other field, utens_stage_out none but possibly utens_stage itself (the
 * very same view).  dtr_stage, beta_v, prec and flags (GTB_WCON_LITERAL,
 * GTB_STATE48) as gtb_vadv.
 * workspace: REQUIRED, at least gtb_vadv_workspace_bytes() bytes, 16-byte
 * aligned, overlapping no field (NULL or too small: GTB_ERR_ARG).
 */
int gtb_step(const gtb_field *in, const gtb_field *coeff, const gtb_field *hdiff_out,
             const gtb_field *u_stage, const gtb_field *wcon, const gtb_field *u_pos,
             const gtb_field *utens, const gtb_field *utens_stage, const gtb_field *utens_stage_out,
             double dtr_stage, double beta_v, int prec, unsigned flags, const int64_t *domain,
             void *workspace, size_t workspace_bytes, void *stream);

/*
 * Batched ensembles of uneven domains (the paper's stencils over many
 * independent members, e.g. an ensemble forecast).  Each member runs
 *   h   = hdiff(in, coeff)                         (gtb_hdiff on its domain)
 *   out = vadv(u_stage = h, wcon, u_pos = h, utens, utens_stage)   (gtb_vadv)
 * A plan validates every member once (the checks of gtb_hdiff and gtb_vadv,
 * plus: h and out may overlap no field of any member, except out being its
 * own member's utens_stage view; in needs 16-byte pitches), builds device
 * tables (one TMA descriptor per member), allocates its scratch and captures
 * a CUDA graph of two persistent kernels (hdiff stage, then vadv stage) that
 * pull work items from atomic queues.  gtb_batch_run replays that graph: it
 * allocates nothing and never synchronises.  A batched member's results equal
 * those of gtb_hdiff + gtb_vadv with the same hdiff tile, bit for bit.  A plan
 * belongs to the device current at creation and holds its members' pointers;
 * runs of one plan must not overlap on the GPU (they share the queues).
 */
typedef struct gtb_member {
    gtb_field in, coeff, h;                   /* hdiff: h = hdiff(in, coeff) */
    gtb_field wcon, utens, utens_stage, out;  /* vadv: out = vadv(h, wcon, h, utens, utens_stage) */
    int64_t domain[3];                        /* (I, J, K), all > 0; K <= 448 */
} gtb_member;

typedef struct gtb_batch_config {
    int32_t hdiff_tile;    /* 0: the single-domain tile (binary64: 4 warps x 16 rows, binary32:
                              8 warps x 8 rows), 1: the other of the two splits */
    int32_t hdiff_levels;  /* K levels per hdiff work item (the K-blocking); <= 0: whole columns */
    int32_t vadv_warps;    /* warps (32 columns each) per vadv work item: 1, 2 or 4 */
    int32_t ctas_per_sm;   /* resident persistent CTAs per SM per stage; <= 0: as many as fit */
} gtb_batch_config;

typedef struct gtb_plan gtb_plan;

int gtb_batch_plan(const gtb_member *members, int n, double dtr_stage, double beta_v, int prec,
                   unsigned flags, const gtb_batch_config *config, gtb_plan **plan);
int gtb_batch_run(const gtb_plan *plan, void *stream);
/* info: hdiff items, vadv items, hdiff grid, vadv grid, total points, members */
int gtb_plan_info(const gtb_plan *plan, int64_t info[6]);
int gtb_plan_destroy(gtb_plan *plan);

/*
 * gtb_vadv_noalloc -- gtb_vadv for callers that cannot allocate device memory.
 * The paper has no counterpart: this exists for code that runs inside a host
 * application that owns every device allocation (a fixed memory budget or a
 * pool it will not hand buffers out of, e.g. a stencil library embedded in a
 * model's time loop) and for latency-critical loops where cudaMalloc's
 * implicit device-wide synchronisation is not acceptable.  Such a caller still
 * passes its inputs and outputs, but no workspace: the forward-sweep state
 * goes to a fixed 16 MiB array inside this library (a file-scope __device__
 * array, held on every GPU that loads the library until the process exits).
 * Same arguments, results and errors as gtb_vadv, plus:
 *  - a domain whose workspace (gtb_vadv_workspace_bytes) exceeds 16 MiB
 *    (1,048,576 points for GTB_F64 storage) is rejected with
 *    GTB_ERR_UNSUPPORTED and nothing is enqueued;
 *  - every call looks up the array's device address in the current device's
 *    context (cudaGetSymbolAddress, which allocates nothing), so a context
 *    that was reset and re-created is never handed a stale address; the
 *    first call on a device may also load the library's kernels there, so
 *    make that first call before any stream capture;
 *  - every call on a device shares the one array, and its contents carry
 *    over between calls (nothing needs to start at zero): calls that may
 *    overlap on the GPU (different streams, or other threads) race and must
 *    be serialised by the caller.
 * No call allocates or frees device memory.
 */
int gtb_vadv_noalloc(const gtb_field *u_stage, const gtb_field *wcon, const gtb_field *u_pos,
                     const gtb_field *utens, const gtb_field *utens_stage,
                     const gtb_field *utens_stage_out, double dtr_stage, double beta_v,
                     int prec, unsigned flags, const int64_t *domain, void *stream);

/*
 * gtb_device_status -- synchronises `stream`, then returns and clears the
 * device error word: GTB_OK, or GTB_ERR_DEVICE if a kernel's bounded wait
 * expired since the last call, or a kernel found a run of addresses outside a
 * field's storage (every kernel of the checked build tests its runs; in the
 * default build the batched column solve does); gtb_last_error() says which.
 * The affected outputs are then unspecified.
 */
int gtb_device_status(void *stream);

/*
 * gtb_selftest_wait -- exercises the bounded-wait failure path that every
 * kernel of the library relies on (the paper has no counterpart): one warp
 * waits on an mbarrier; with arrive = 0 nobody completes it, the wait gives up
 * after limit_ns (0 < limit_ns <= 2e9), sets the device error word and the
 * kernel returns, so that gtb_device_status() then reports GTB_ERR_DEVICE and
 * the context stays usable; with arrive = 1 one thread completes the phase
 * first and nothing is reported.  Bad arguments: GTB_ERR_ARG.
 */
int gtb_selftest_wait(long long limit_ns, int arrive, void *stream);

/*
 * gtb_probe_fp64_fma -- a measurement kernel, not a step of the method (the
 * paper has no counterpart): `blocks` CTAs of 256 threads, each thread running
 * 8 independent binary64 FMA chains of `iters` FMAs, i.e. blocks * 256 * 8 *
 * iters FMA instructions.  Timed by the caller (CUDA events on `stream`), it
 * gives the GPU's FP64 FMA issue rate, the peak that the binary64 column solve
 * is reported against.  `sink`: 8 bytes of device memory, never written in
 * practice.  Bad arguments: GTB_ERR_ARG / GTB_ERR_NULL / GTB_ERR_LAYOUT.
 */
int gtb_probe_fp64_fma(int blocks, int iters, void *sink, void *stream);

/* Message for the last failed call on this thread ("" if none). */
const char *gtb_last_error(void);

/* Library version string, e.g. "gtb 0.2 sm_103a". */
const char *gtb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GTB_H */
