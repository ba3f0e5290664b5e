/*
 * rtproj.h -- C ABI of the GB300 (sm_103a) randomized orthogonal projection library.
 *
 * Method: Rokhlin & Tygert, "A fast randomized algorithm for orthogonal projection"
 * (arXiv 0912.1135). For a full-rank real m x n matrix A (m <= n) the library
 * computes, for blocks of right-hand sides b,
 *   - the projection onto the null space of A, Zb = b - A^*(AA^*)^{-1}Ab   (Eq. 1),
 *     through the preconditioned form of Eq. 11;
 *   - the projection onto the row space, A^* h;
 *   - the least-squares solution h = argmin ||A^* h - b||                 (Remark 4.1).
 * The preconditioner P = Pi^* R^* comes from a pivoted QR of the sketch S = A G
 * (Eqs. 12-13), G an n x l random matrix generated on the device and never stored.
 *
 * Conventions (all functions):
 *   - Matrices are row-major. A, the right-hand sides and the outputs of the apply are
 *     float64, or float32 when the handle was created with opts.dtype = RTPROJ_F32 (they
 *     are then passed as void*; every internal quantity stays float64 and float32 input is
 *     widened exactly). A is m x n with leading dimension lda >= n (in elements).
 *     Right-hand sides are stored as ROWS: B is k x n (row j is the j-th vector b),
 *     ldb >= n; null/row-space outputs are k x n; least-squares outputs are k x m.
 *   - Pointers named A, B, Z, ROW, H, S, workspace are DEVICE pointers unless the
 *     comment says otherwise. The library never allocates device memory: all
 *     scratch lives in the caller's workspace. It never frees caller memory.
 *   - A is borrowed: it must stay alive and unchanged from rtproj_create until
 *     rtproj_destroy (or the next rtproj_create on the same memory).
 *   - All work is enqueued on the stream given to rtproj_create (a cudaStream_t
 *     passed as void*; NULL means the legacy default stream). Calls are
 *     asynchronous except rtproj_precondition, rtproj_get_info, rtproj_export_state
 *     and rtproj_sketch, which synchronize that stream once, rtproj_create in the
 *     mixed mode, which waits for the slicing of A to learn whether A held non-finite
 *     entries, and the apply calls when opts.refine_tol > 0, which read the size of
 *     each refinement correction back to decide whether to stop.
 *   - Errors: invalid arguments return immediately with a status and enqueue
 *     nothing. Conditions found on the device (rank deficiency, Cholesky breakdown,
 *     non-finite values, an expired bounded wait) are latched in a device status
 *     word; rtproj_precondition returns it, and rtproj_get_info reports it for
 *     the apply calls. No kernel traps, asserts or waits without a bound.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef RTPROJ_H
#define RTPROJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtproj_ctx* rtproj_t;

typedef enum {
    RTPROJ_OK = 0,
    RTPROJ_EINVAL = 1,       /* invalid argument: sizes, leading dimensions, null pointer */
    RTPROJ_ESTATE = 2,       /* apply called before a successful rtproj_precondition      */
    RTPROJ_ERANK = 3,        /* |R_mm| <= rank_tol * |R_11| after the pivoted QR of S^*:
                                A G is numerically rank deficient (Lemma 2.4 needs full rank) */
    RTPROJ_ENOTSPD = 4,      /* Cholesky of X = P^{-1} A A^* P^{-*} broke down            */
    RTPROJ_ENONFINITE = 5,   /* a NaN or infinity reached the factorizations             */
    RTPROJ_ETIMEOUT = 6,     /* a bounded device-side wait gave up                        */
    RTPROJ_ENOMEM = 7,       /* workspace smaller than rtproj_workspace_bytes(), or (for
                                rtproj_sketch_noalloc) m * l above its fixed scratch array */
    RTPROJ_ECUDA = 8,        /* a CUDA runtime call failed                                */
    RTPROJ_EUNSUPPORTED = 9  /* option combination not supported                          */
} rtproj_status;

/* Arithmetic of the whole path. */
typedef enum {
    /* Every product in float64 on the FP64 pipe (the plain float64 form). */
    RTPROJ_PLAIN_FP64 = 0,
    /* Products with A on the bfloat16 tensor cores through exact fixed-point slicing
       (each operand split into s bfloat16 slices of 8 bits; slice products summed
       exactly in float32 and combined in 64-bit integers), a low-slice sketch,
       and one or more refinement passes (Remark 4.3) whose residuals carry more
       than float64 accuracy. The pivoted QR (qr_form), R^{-*} and the Cholesky factor
       of X run in float-float on the FP32 pipe, each with the float64 kernel enqueued
       behind it for ranges float-float cannot hold; T1 = L^{-1} R^{-*} is formed in
       float64, and the m x m stage's products with it are sliced tensor-core products
       (apply_slices). */
    RTPROJ_MIXED_REFINED = 1
} rtproj_mode;

/* Element type of A, the right-hand sides and the apply's outputs. */
typedef enum {
    RTPROJ_F64 = 0,
    RTPROJ_F32 = 1
} rtproj_dtype;

/* Distribution of the entries of G (Eq. 12), from Philox4x32-10 (Salmon, Moraes, Dror &
   Shaw, SC'11) with key (seed mod 2^32, seed >> 32).
   UNIFORM and RADEMACHER: entry (i, j) takes byte u = byte (i & 3) of word
   ((i & 15) >> 2) of the block at counter (i >> 4, j, 0, 0).
   GAUSSIAN: entries 4q .. 4q+3 of column j come from the block (x, y, z, w) at counter
   (q, j, 1, 0) by the Box-Muller transform (Box & Muller, Ann. Math. Stat. 1958) in
   float32: u1 = ((x >> 9) + 1/2) 2^-23, u2 = (y >> 9) 2^-23, r = sqrt(-2 ln u1),
   entries 4q and 4q+1 are r cos(2 pi u2) and r sin(2 pi u2), and (z, w) give 4q+2 and
   4q+3 the same way; each variate is then rounded to the nearest multiple of 2^-12
   (ties to even), so |G_ij| < 5.78 and every entry is exact in two bfloat16 digits. */
typedef enum {
    RTPROJ_OMEGA_UNIFORM = 0,     /* (2u - 255)/256: uniform on (-1,1), as in Tables 1, 2, 5, 6 */
    RTPROJ_OMEGA_RADEMACHER = 1,  /* +1 if u >= 128 else -1                                    */
    RTPROJ_OMEGA_GAUSSIAN = 2     /* standard normal (Section 3, Theorem 3.1; Tables 3, 4)     */
} rtproj_omega;

typedef struct {
    int mode;            /* rtproj_mode (default RTPROJ_MIXED_REFINED)                    */
    int omega;           /* rtproj_omega (default RTPROJ_OMEGA_GAUSSIAN)                  */
    int sketch_slices;   /* mixed: slices of A in S = A G            (default 5, 1..10)  */
    int gram_slices;     /* mixed: slices in W = P^{-1} A            (default 7, 1..10)  */
    int gram2_slices;    /* mixed: slices in X = W W^*               (default 4, 1..10)  */
    int apply_slices;    /* mixed: slices in c = A b and A^* dh      (default 7, 1..10)  */
    int resid_slices;    /* mixed: slices in the refinement residual (default 9, 1..10)  */
    int refine_passes;   /* mixed: refinement passes (default 1, 0..8); with refine_tol > 0
                            the largest number of passes                                 */
    int timing;          /* 1: record CUDA events around each phase (rtproj_get_timings)  */
    double rank_tol;     /* ERANK threshold; <= 0 selects 8 u, u the sketch's relative
                            precision: 2^-52 in the float64 and sparse forms, 2^(-8 s) for
                            the mixed form's s = sketch_slices digits of A              */
    int dtype;           /* rtproj_dtype of A, B and the outputs (default RTPROJ_F64)     */
    long long spin_limit_cycles;  /* bound, in SM clock cycles, on each grid-exchange wait of
                            the pivoted QR and the Cholesky (default 4e9, about 2 s); when it
                            expires the kernel latches RTPROJ_ETIMEOUT and every CTA returns.
                            The tensor-core products keep their own fixed bound.          */
    double refine_tol;   /* mixed: refine until the correction dh of every right-hand side
                            satisfies ||dh|| <= refine_tol max(||h||, ||b|| / ||A||_F)
                            (Remark 4.3), at most refine_passes passes; 0 (default) runs
                            exactly refine_passes                                         */
    int scalable;        /* 1: reserve what rtproj_set_scaling needs (the float64 form keeps
                            A diag(d) in the workspace; the mixed form forms it in the Gram
                            matrix's buffer and needs nothing more). Default 0.             */
    int qr_form;         /* mixed form's pivoted QR: 0 (default) float-float on the whole
                            grid (one grid exchange per step, the column updates on the FP32
                            pipe); 1 float-float on one 16-CTA cluster (exchange through
                            distributed shared memory) when S^* fits its shared memory, else
                            2; 2 the float64 kernel of the float64 form. Forms 0 and 1 fall
                            back to 2 by themselves when the entries' range would take
                            float-float near float's underflow. All give a valid pivoted
                            QR; the preconditioner tolerates float-float's 2^-48 and the
                            refinement makes the projection exact.                      */
    int async;           /* 1: rtproj_create and rtproj_precondition do not synchronize; the
                            conditions they would return (non-finite A, ERANK, ENOTSPD,
                            ETIMEOUT) stay latched in the device status word, which
                            rtproj_get_info reports, and the apply runs regardless. Lets a
                            serving loop overlap consecutive steps and lets precondition and
                            the apply be captured in a CUDA graph (with refine_tol = 0).
                            Default 0.                                                    */
} rtproj_opts;

/* Phases timed when opts.timing is set (indices into rtproj_get_timings' arrays). */
typedef enum {
    RTPROJ_PHASE_SKETCH = 0,    /* S = A G (Eq. 12), Omega generation included        */
    RTPROJ_PHASE_QR = 1,        /* pivoted QR of S^* (Eq. 13)                          */
    RTPROJ_PHASE_GRAM = 2,      /* W = P^{-1} A and X = W W^* (Eq. 14, steps a-e)      */
    RTPROJ_PHASE_FACTOR = 3,    /* R^{-*}, Cholesky of X, T1 = L^{-1} R^{-*}           */
    RTPROJ_PHASE_APPLY_A = 4,   /* reductions over n: c = A b, r = A s                 */
    RTPROJ_PHASE_APPLY_M = 5,   /* the m x m stage (steps 2-6)                         */
    RTPROJ_PHASE_APPLY_AT = 6,  /* products with A^*: b - A^* h, row = A^* h           */
    RTPROJ_PHASE_SLICE = 7,     /* mixed mode: slicing of operands into bfloat16 planes */
    RTPROJ_NUM_PHASES = 8
} rtproj_phase;

typedef struct {
    int status;              /* latched device status (an rtproj_status value)            */
    int preconditioned;      /* 1 after a successful rtproj_precondition                  */
    int64_t m, n, l;
    double r11, rmm;         /* |R_11| and |R_mm| of the pivoted QR of S^*                */
    double l11, lmm;         /* largest and smallest diagonal entries of chol(X)          */
    float ms_precondition;   /* device time of the last rtproj_precondition (ms)          */
    double kappa_R;          /* r11 / rmm: estimates kappa(A G), about kappa(A) (Lemma 2.4) */
    double kappa_pre;        /* l11 / lmm: lower estimate of kappa(P^{-1} A) = kappa(X)^(1/2) */
    double norm_A;           /* ||A||_F, computed at create                               */
    double resid_rel;        /* mixed form, last apply: max over right-hand sides of
                                ||A s|| / (||A||_F ||b||) for the s that entered the last
                                refinement pass (Section 5's delta, normalised); 0 when no
                                pass ran                                                  */
    double dh_rel;           /* mixed form, last apply: max over right-hand sides of
                                ||dh|| / max(||h||, ||b|| / ||A||_F) for the last refinement
                                correction dh (||A||_F ||dh|| bounds its change to Zb)     */
    int passes;              /* refinement passes run by the last apply                   */
} rtproj_info;

/* Fills *opts with the defaults listed above. */
void rtproj_default_opts(rtproj_opts* opts);

/* Device workspace (bytes) needed for an m x n matrix, sketches with l <= l_max and
   applies with k <= k_max right-hand sides, under opts (NULL: defaults). Returns 0
   for invalid sizes. The workspace must be 256-byte aligned. */
size_t rtproj_workspace_bytes(int64_t m, int64_t n, int64_t l_max, int64_t k_max,
                              const rtproj_opts* opts);

/* Creates a handle bound to the device matrix A (m x n, row-major, lda >= n, 1 <= m <= n),
   the caller's device workspace and stream. In the mixed mode it also slices A into
   bfloat16 slice planes, in both the row-major and the transposed layout (kept in the
   workspace), and synchronizes the stream once; the later calls of that mode read only
   the planes. The current CUDA device must be the one that holds A and the workspace. */
rtproj_status rtproj_create(rtproj_t* out, int64_t m, int64_t n, const void* A, int64_t lda,
                            int64_t l_max, int64_t k_max, void* workspace, size_t ws_bytes,
                            void* stream, const rtproj_opts* opts);

/* A sparse A, optionally plus a low-rank term: A = S + U V (Section 5: the sparse test
   matrix of Eq. 21 and its sum with a rank-10 term, Eq. 22). S is m x n in compressed
   sparse row form on the device: row_ptr (m + 1 int64, row_ptr[0] = 0, non-decreasing,
   row_ptr[m] = nnz), col_idx (nnz int32 in [0, n), any order within a row, duplicates
   summed) and val (nnz float64). U (m x r, row-major, ld r) and V (r x n, row-major,
   ld n) are float64 device matrices, r = 0 (U, V null) for S alone, 0 <= r <= min(m, 64);
   k_max <= 65535.
   All of them are borrowed: they must stay alive and unchanged until rtproj_destroy.
   The handle runs the float64 arithmetic of the dense float64 form on the products that
   build the preconditioner (S_k = A G with G generated per nonzero; X column by column
   as in steps a-e after Eq. 15: D = A^* P^-, E = A D, X = R^{-*} Pi E) and sums every
   product with A or A^* of the apply and its refinement passes (Remark 4.3; opts
   refine_passes and refine_tol) in double-double, so that the refinement converges to
   the projection of the stored matrix. A product with A costs O(nnz + r (m + n)).
   opts.mode, the slice counts and qr_form do not apply; dtype must be RTPROJ_F64 and
   scalable 0 (else RTPROJ_EUNSUPPORTED). rtproj_create_sparse synchronizes the stream:
   it reads row_ptr on the host (RTPROJ_EINVAL if malformed), builds a column-compressed
   copy in the workspace and checks col_idx (RTPROJ_EINVAL) and val, U, V
   (RTPROJ_ENONFINITE) on the device. The later calls are those of a dense handle
   (precondition, the applies, sketch, get_info, export_state, destroy); set_scaling
   returns RTPROJ_EUNSUPPORTED. */
size_t rtproj_sparse_workspace_bytes(int64_t m, int64_t n, int64_t nnz, int64_t r, int64_t l_max,
                                     int64_t k_max, const rtproj_opts* opts);
rtproj_status rtproj_create_sparse(rtproj_t* out, int64_t m, int64_t n, int64_t nnz,
                                   const int64_t* row_ptr, const int32_t* col_idx,
                                   const double* val, int64_t r, const double* U,
                                   const double* V, int64_t l_max, int64_t k_max,
                                   void* workspace, size_t ws_bytes, void* stream,
                                   const rtproj_opts* opts);

/* Builds the preconditioner from seed and l (m <= l <= min(n, l_max); Section 4):
   the sketch S = A G (Eq. 12), the pivoted QR S^* = Q R Pi (Eq. 13), and the Gram
   matrix X = P^{-1} A A^* P^{-*} (Eq. 14, steps a-e) factored by Cholesky in place of
   the explicit inverse Y = X^{-1} of Eq. 16. Synchronizes the stream once and returns
   the latched device status (RTPROJ_ERANK, RTPROJ_ENOTSPD, RTPROJ_ENONFINITE). */
rtproj_status rtproj_precondition(rtproj_t h, uint64_t seed, int64_t l);   /* see opts.async */

/* Null-space projection (Eq. 11; the seven steps of Section 4, then b - b~):
   Z = rows of Zb for the k rows of B (k <= k_max). Z may alias B exactly
   (Z == B, ldz == ldb) but must not partially overlap it. */
rtproj_status rtproj_null_project(rtproj_t h, const void* B, int64_t ldb, int64_t k,
                                  void* Z, int64_t ldz);

/* Row-space projection b~ = A^* h (step 7 of Section 4), k x n into ROW. */
rtproj_status rtproj_row_project(rtproj_t h, const void* B, int64_t ldb, int64_t k,
                                 void* ROW, int64_t ldr);

/* Least-squares solutions h = argmin ||A^* h - b|| (Remark 4.1), k x m into X. */
rtproj_status rtproj_lstsq(rtproj_t h, const void* B, int64_t ldb, int64_t k,
                           void* X, int64_t ldx);

/* All three outputs of one apply; any output pointer may be NULL. */
rtproj_status rtproj_project(rtproj_t h, const void* B, int64_t ldb, int64_t k,
                             void* Z, int64_t ldz, void* ROW, int64_t ldr,
                             void* X, int64_t ldx);

/* Sketch only: S = A G (Eq. 12) into the device buffer S (m x l, row-major, lds >= l),
   in the handle's mode (float64 products, or sketch_slices bfloat16 slices of A).
   Synchronizes. Used to test the sketch step on its own. */
rtproj_status rtproj_sketch(rtproj_t h, uint64_t seed, int64_t l, double* S, int64_t lds);

/* The float64 sketch S = A G of rtproj_sketch, for callers that cannot allocate device
   memory: applications whose device memory is owned by a pooling allocator or a fixed
   budget (a cudaMalloc would fail or fragment the pool), and loops that cannot afford the
   device synchronization cudaMalloc implies. The paper has no counterpart: it is a
   packaging of the sketch that needs no workspace.
   A (m x n, row-major, lda >= n) and S (m x l, row-major, lds >= l) are device pointers,
   m <= l <= n; omega is an rtproj_omega value; stream is a cudaStream_t passed as void*
   and must belong to the current device (RTPROJ_EINVAL otherwise).
   The split-K scratch is a fixed array inside the library: 32 MiB of device memory
   (4 Mi float64 entries), held on every GPU that loads the library until the process
   exits. Nothing is allocated. Returns RTPROJ_ENOMEM when m * l exceeds 4 Mi entries and
   RTPROJ_EINVAL for invalid sizes; asynchronous otherwise. The first call on a device
   looks up the array's device address (with that device current): make it before any
   stream capture. Every call shares the array and overwrites what it reads from it;
   calls that overlap on the GPU race on it, so serialize them. */
rtproj_status rtproj_sketch_noalloc(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed,
                                    int64_t l, int omega, double* S, int64_t lds, void* stream);

/* The test matrix G of Eq. 12 itself: entries G[i][j] (i < n, j < l) of distribution
   omega (an rtproj_omega value) for seed, written as float64 into the device buffer G
   (n x l, row-major, ldg >= l) on stream (a cudaStream_t passed as void*). The sketch
   never stores G; this entry point exists to check step a1 on its own. Asynchronous;
   RTPROJ_EINVAL for invalid arguments. */
rtproj_status rtproj_generate_omega(uint64_t seed, int64_t n, int64_t l, int omega, double* G, int64_t ldg, void* stream);

/* Gradient with respect to A of L = sum_j <g_j, Z b_j> (the adjoint of Eq. 1; the paper
   does not differentiate, this follows from it): with P = A^*(AA^*)^{-1},
   dZ = -(Z dA^* P^* + P dA Z), so dL/db_j = Z g_j and
       dL/dA = -sum_j (h_j (Z g_j)^* + w_j (Z b_j)^*) = -(H^* Y + W^* Zb),
   where h_j = lstsq(b_j) and w_j = lstsq(g_j) (Remark 4.1). Inputs are k x m (H, W: rows
   h_j, w_j) and k x n (Y: rows Z g_j; Zb: rows Z b_j), all in the handle's element type
   and on its device, as rtproj_project returns them; dA is m x n (ldda >= n). The product
   runs in the handle's mode (digit-sliced tensor-core products with apply_slices digits, or
   float64). workspace: device, 256-byte aligned, at least rtproj_grad_workspace_bytes(h, k)
   bytes, caller-owned. Asynchronous on the handle's stream. */
size_t rtproj_grad_workspace_bytes(rtproj_t h, int64_t k);
rtproj_status rtproj_grad_A(rtproj_t h, int64_t k, const void* H, int64_t ldh, const void* Y, int64_t ldy,
                            const void* W, int64_t ldw, const void* Zb, int64_t ldz, void* dA, int64_t ldda,
                            void* workspace, size_t ws_bytes);

/* Interior-point-style column scaling: from now on the handle's matrix is A diag(d), with
   A the matrix given to rtproj_create (still borrowed) and d a DEVICE array of n float64
   scalings (NULL restores A). The scaled matrix is formed on the device (each entry's
   product rounded once), its Frobenius norm recomputed and, in the mixed form, sliced
   again into both digit layouts; the preconditioner is dropped (call rtproj_precondition
   next). Needs opts.scalable = 1 at create. Synchronizes like rtproj_create unless
   opts.async; d is read on the handle's stream. */
rtproj_status rtproj_set_scaling(rtproj_t h, const double* d);

/* Replaces the handle's spin_limit_cycles (see rtproj_opts) for later calls; cycles >= 1. */
rtproj_status rtproj_set_spin_limit(rtproj_t h, long long cycles);

/* Copies the preconditioner state to HOST buffers (any may be NULL): R (m x m,
   row-major, upper triangular), perm (m entries: position j of the pivoted QR holds
   original column perm[j] of S^*, so (Pi x)[j] = x[perm[j]]), and Lc (m x m, the
   lower-triangular Cholesky factor of X). Synchronizes. */
rtproj_status rtproj_export_state(rtproj_t h, double* R, int32_t* perm, double* Lc);

/* Synchronizes, then returns per phase the device milliseconds (ms[p]) and the number
   of timed occurrences (count[p]) accumulated since the previous call, and resets them.
   Arrays have RTPROJ_NUM_PHASES entries; either may be NULL. Needs opts.timing = 1. */
rtproj_status rtproj_get_timings(rtproj_t h, double* ms, int64_t* count);

/* Number of kernels this library has enqueued since it was loaded (all handles). */
uint64_t rtproj_launch_count(void);

/* Synchronizes the stream and reports the latched status and diagnostics. */
rtproj_status rtproj_get_info(rtproj_t h, rtproj_info* info);

/* Clears the latched device status (after the caller handled it). */
rtproj_status rtproj_clear_status(rtproj_t h);

/* Releases the host-side handle. Does not touch A or the workspace. */
rtproj_status rtproj_destroy(rtproj_t h);

/* Static string for a status code. */
const char* rtproj_status_string(rtproj_status s);

#ifdef __cplusplus
}
#endif

#endif /* RTPROJ_H */
