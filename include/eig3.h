/*
 * eig3.h -- C ABI of the GB300 (sm_103a) library for batched, numerically
 * stable closed-form eigenvalues of real diagonalizable 3x3 matrices.
 *
 * Method: Habera & Zilian, "Numerically stable evaluation of closed-form
 * expressions for eigenvalues of 3x3 matrices" (arXiv 2511.00292):
 *   I1 (Algorithm 1) -> J2 (Algorithm 2) -> J3 (Algorithm 4)
 *   -> Delta (Algorithm 5, sum of products) -> eigenvalues (Algorithm 6,
 *   trigonometric formula with the arctangent triple angle, Eq. for phi).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are pointers the current CUDA device can access:
 *    device memory (cudaMalloc, a torch CUDA tensor), or page-locked host
 *    memory (cudaHostAlloc / cudaHostRegister), which the kernels then read
 *    and write directly over the host link, with no staging copy.  Pageable
 *    host memory is not allowed.  The caller owns every buffer; the library
 *    never allocates, frees or synchronises.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL means the legacy default stream).  The returned status covers the
 *    host-side argument checks and the launch (cudaGetLastError); errors of
 *    the kernel itself surface at the caller's next synchronisation.
 *  - Calls hold no host state between launches and read nothing back, so a
 *    sequence of calls can be captured into a CUDA graph.
 *  - n == 0 returns EIG3_OK without launching.  n < 0 or a NULL required
 *    pointer with n > 0 returns EIG3_ERR_ARG; nothing is launched.
 *  - Every pointer must be aligned to its element size (8 bytes for FP64,
 *    4 for FP32), else EIG3_ERR_ALIGN.  Rows are packed: matrix i starts at
 *    element 9*i (EIG3_GENERAL9) or 6*i (EIG3_SYM6).
 *  - Non-finite input entries give non-finite outputs for that matrix; no
 *    kernel traps.
 *
 * Layouts (`layout`)
 *  EIG3_GENERAL9  row-major A00 A01 A02 A10 A11 A12 A20 A21 A22, 0-based
 *                 indices as in the paper (Section "Invariant I1").
 *  EIG3_SYM6      symmetric matrix stored as A00 A11 A22 A12 A02 A01 (Voigt
 *                 order; the paper's symmetric routine does not fix one).
 *
 * Storage type (`dtype`) and arithmetic (`precision`)
 *  EIG3_F64 + EIG3_PREC_F64        binary64 in, binary64 arithmetic, binary64 out.
 *  EIG3_F32 + EIG3_PREC_F64        binary32 in, binary64 arithmetic, binary32 out.
 *  EIG3_F32 + EIG3_PREC_F32_COMP   binary32 in, binary32 compensated arithmetic
 *                                  (error-free TwoSum/TwoProduct transformations,
 *                                  per-matrix power-of-two scaling of the
 *                                  deviatoric part), binary32 out.  The
 *                                  invariants output is accumulated by Sum2
 *                                  (accurate at u32^2); the eigenvalues of
 *                                  symmetric input take the invariants from
 *                                  sums on a fixed grid, accurate to the
 *                                  absolute level the triple angle needs.  No
 *                                  binary64 arithmetic on this path except the
 *                                  binary64 invariants output of
 *                                  eig3_invariants.
 *  EIG3_F32 + EIG3_PREC_F32_COMP_A64
 *                                  as EIG3_PREC_F32_COMP, except that the final
 *                                  combination of the compensated Delta and
 *                                  27 J3 and the triple angle of Algorithm 6
 *                                  are taken in binary64 for every matrix (the
 *                                  sines rounded back to binary32).  It is
 *                                  the upper end of any rule that takes these
 *                                  steps in binary64 below a Delta/J2^3
 *                                  threshold, and measures what binary64
 *                                  there can buy.  Accepted by
 *                                  eig3_eigvals and eig3_eigvals_backward (the
 *                                  adjoint is the EIG3_PREC_F32_COMP one); the
 *                                  other entry points reject it with
 *                                  EIG3_ERR_DTYPE.
 *  EIG3_F64 + EIG3_PREC_F32_COMP or EIG3_PREC_F32_COMP_A64
 *                                  rejected with EIG3_ERR_DTYPE.
 *  EIG3_F64/F32 + EIG3_PREC_F64_GUARDED
 *                                  binary64 arithmetic with a guard for
 *                                  ill-conditioned eigenbases (where Sections
 *                                  J3, Delta and Eigenvalues find Algorithms 4
 *                                  and 5 lose accuracy and an iterative method
 *                                  does not): a general matrix whose deviatoric
 *                                  part S is far from normal, ||S||_F^2 >
 *                                  32 tr(S^2), gets its eigenvalues from the
 *                                  shifted QR algorithm on the 3x3 matrix
 *                                  (backward stable, at most 64 steps); every
 *                                  other matrix gets exactly the
 *                                  EIG3_PREC_F64 results.  Symmetric input
 *                                  (normal) is never switched.  Accepted by
 *                                  eig3_eigvals and eig3_eigvals_backward;
 *                                  the other entry points reject it with
 *                                  EIG3_ERR_DTYPE.
 *
 * Readings of the paper built into the library
 *  - Algorithm 5, term r10: +M02*M21*d2 (the printed minus sign does not
 *    reproduce the discriminant 4 J2^3 - 27 J3^2).
 *  - Algorithm 6: phi = atan2(sqrt(27 Delta), 27 J3), in [0, pi].
 *  - Computed J2 < 0 or Delta < 0 (possible for nonsymmetric input) are
 *    clamped to 0 before the square roots.
 *  - Output eigenvalues are ascending, lambda_1 <= lambda_2 <= lambda_3
 *    (the ordering of the trigonometric formula, Section 1).
 */
#ifndef EIG3_H
#define EIG3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EIG3_OK = 0,
  EIG3_ERR_ARG = 1,    /* n < 0, a required pointer is NULL while n > 0, or a
                          scalar argument (material constant, variant) is out
                          of its range                                           */
  EIG3_ERR_LAYOUT = 2, /* layout is not EIG3_GENERAL9 or EIG3_SYM6              */
  EIG3_ERR_DTYPE = 3,  /* unsupported dtype / precision combination             */
  EIG3_ERR_ALIGN = 4,  /* a pointer is not aligned to its element size          */
  EIG3_ERR_CUDA = 5    /* the launch failed (cudaGetLastError after the launch) */
} eig3_status;

enum { EIG3_GENERAL9 = 0, EIG3_SYM6 = 1 };
enum { EIG3_F64 = 0, EIG3_F32 = 1 };
enum {
  EIG3_PREC_F64 = 0,
  EIG3_PREC_F32_COMP = 1,
  EIG3_PREC_F64_GUARDED = 2,
  EIG3_PREC_F32_COMP_A64 = 3
};
/* Invariant evaluations of eig3_eigvals_variant (the paper's comparisons). */
enum { EIG3_VARIANT_PRESENT = 0, EIG3_VARIANT_NAIVE = 1, EIG3_VARIANT_NAIVE_TENSOR = 2 };

/*
 * Per-launch numerical statistics, accumulated on the device by
 * eig3_eigvals when a non-NULL device pointer is passed.  Reset it with
 * eig3_stats_reset before the first accumulating call.  48 bytes, 8-aligned.
 * Several calls may accumulate into one struct (counts add, min/max combine).
 */
typedef struct {
  unsigned long long n_delta_clamped; /* matrices whose computed Delta was < 0     */
  unsigned long long n_j2_clamped;    /* matrices whose computed J2 was < 0        */
  unsigned long long n_nonfinite;     /* matrices with a non-finite eigenvalue      */
  double min_disc_ratio;              /* min over matrices with J2 > 0 of
                                         Delta+/J2+^3 = 4 sin^2(phi), in [0, 4]
                                         (0 at a repeated eigenvalue); evaluated in
                                         binary32 from the computed triple angle */
  double max_abs_lambda;              /* max over matrices of max_k |lambda_k|      */
  unsigned long long n_guarded;       /* matrices EIG3_PREC_F64_GUARDED switched to
                                         the QR algorithm                           */
} eig3_stats;

/*
 * eig3_invariants -- the four invariants of Algorithms 1, 2, 4 and 5.
 *   A    device, n matrices in `layout` / `dtype` (read only).
 *   inv  device, n x 4 binary64, row i = (I1, J2, J3, Delta) of matrix i,
 *        before any clamping (Delta may be slightly negative for
 *        nonsymmetric input).  With EIG3_PREC_F32_COMP the compensated
 *        binary32 values are returned unscaled in binary64.
 */
eig3_status eig3_invariants(const void *A, int layout, int dtype, int precision, int64_t n,
                            double *inv, void *stream);

/*
 * eig3_eigvals -- ascending eigenvalues by Algorithm 6 on the stable invariants.
 *   A      device, n matrices (read only).
 *   lam    device, n x 3 of `dtype`: (lambda_1, lambda_2, lambda_3) per matrix.
 *   aux    device, n x 4 of `dtype`, or NULL.  When given, receives the
 *          values the adjoint needs, (r, sigma_1, sigma_2, I1) with
 *          r = sqrt(3 J2+), sigma_1 = sin(phi/3), sigma_2 = sin((pi-phi)/3);
 *          pass it back to eig3_eigvals_backward to skip the recomputation.
 *          For a matrix that EIG3_PREC_F64_GUARDED switched to the QR
 *          algorithm the same quantities follow from its eigenvalue gaps:
 *          r^2 = g12^2 + g12 g23 + g23^2, sigma_1 = (sqrt3/2) g12 / r,
 *          sigma_2 = (sqrt3/2) g23 / r (g12 = lambda_2 - lambda_1,
 *          g23 = lambda_3 - lambda_2), and I1 is the trace.
 *   stats  device eig3_stats or NULL (see eig3_stats_reset).
 */
eig3_status eig3_eigvals(const void *A, int layout, int dtype, int precision, int64_t n,
                         void *lam, void *aux, eig3_stats *stats, void *stream);

/*
 * eig3_eigvals_backward -- vector-Jacobian product of eig3_eigvals.
 * Given grad_lam (dL/dlambda_k, n x 3 of `dtype`), writes
 *   grad_A = dL/dA = a_I1 I + a_J2 dev(A)^T + a_J3 dev(cof(dev A))
 * with a_I1 = sum_k g_k / 3 and (a_J2, a_J3) from the chain rule through the
 * trigonometric formula (Jacobians of J2 and J3: Lemmas of Sections J2 and
 * J3).  For EIG3_SYM6 the gradient is taken with respect to the six stored
 * entries (an off-diagonal entry stands for both A_ij and A_ji, so it gets
 * G_ij + G_ji).  Where two computed eigenvalues coincide exactly the
 * individual eigenvalues are not differentiable; the weights of such a
 * cluster are then replaced by their mean (the gradient of the cluster sum).
 *   A         device, n matrices (read only).
 *   grad_lam  device, n x 3 of `dtype` (read only).
 *   aux       device n x 4 from eig3_eigvals on the same A, or NULL to
 *             recompute it.
 *   grad_A    device, n x 9 or n x 6 of `dtype`.
 */
eig3_status eig3_eigvals_backward(const void *A, int layout, int dtype, int precision, int64_t n,
                                  const void *grad_lam, const void *aux, void *grad_A,
                                  void *stream);

/*
 * eig3_eigvals_vjp -- the eigenvalues and the gradient of a loss linear in
 * them, L = sum_k w_k lambda_k, in one pass per matrix: the forward of
 * eig3_eigvals (Algorithms 1, 2, 4, 5, 6) followed by the vector-Jacobian
 * product of eig3_eigvals_backward with the weights w, with no adjoint inputs
 * written or read back.  The gradient is the same quantity,
 *   grad_A = a_I1 I + a_J2 dev(A)^T + a_J3 dev(cof(dev A))
 * (Jacobians of J2 and J3: Lemmas of Sections J2 and J3; the chain rule
 * through Algorithm 6), with the same layout convention for EIG3_SYM6 and the
 * same cluster-mean rule where two computed eigenvalues coincide exactly; it
 * is evaluated on the scaled deviatoric data and reuses the products of the
 * invariants, so it agrees with eig3_eigvals_backward to rounding, not bit
 * for bit.  The eigenvalues are those of eig3_eigvals bit for bit.  For a
 * loss that is not linear in lambda use eig3_eigvals + eig3_eigvals_backward
 * (the weights are then dL/dlambda, which depend on lambda).
 *   A       device, n matrices (read only).
 *   w       device, n x 3 of `dtype`: w_k of matrix i at w[3 i + k - 1] (read only).
 *   lam     device, n x 3 of `dtype` (ascending eigenvalues), or NULL.
 *   grad_A  device, n x 9 or n x 6 of `dtype`.
 *   stats   device eig3_stats or NULL (as for eig3_eigvals).
 * Precisions EIG3_PREC_F64 (EIG3_F64 or EIG3_F32 storage) and
 * EIG3_PREC_F32_COMP (EIG3_F32); the others return EIG3_ERR_DTYPE.
 */
eig3_status eig3_eigvals_vjp(const void *A, int layout, int dtype, int precision, int64_t n,
                             const void *w, void *lam, void *grad_A, eig3_stats *stats,
                             void *stream);

/*
 * eig3_eigprojectors -- eigenvalues and eigenprojectors E_1, E_2, E_3.
 * Section 1 of the paper relates the eigenprojectors to the eigenvalue
 * derivatives, E_k^T = d lambda_k / dA; with the Jacobians of J2 and J3
 * (Lemmas of Sections J2 and J3) this gives
 *   E_k = I/3 + a_J2(k) dev(A) + a_J3(k) dev(cof(dev A))^T,
 * with (a_J2(k), a_J3(k)) the adjoint scalars of eig3_eigvals_backward for
 * the weights e_k.  sum_k E_k = I, E_j E_k = delta_jk E_k and A E_k = lambda_k E_k
 * for distinct eigenvalues.  Where two computed eigenvalues coincide exactly
 * each of them gets half the projector onto their joint eigenspace (the
 * cluster-mean convention of the adjoint).
 *   A    device, n matrices (read only).
 *   lam  device, n x 3 of `dtype` (ascending eigenvalues), or NULL.
 *   P    device, n x 3 x 9 of `dtype`: P[27 i + 9 k + 3 r + c] = (E_{k+1})_{rc}
 *        of matrix i (row-major 3 x 3, also for EIG3_SYM6 input).
 */
eig3_status eig3_eigprojectors(const void *A, int layout, int dtype, int precision, int64_t n,
                               void *lam, void *P, void *stream);

/*
 * eig3_mohr_coulomb -- Mohr-Coulomb yield function of the stress tensors
 * sigma and, optionally, its gradient (Section "Application"):
 *   f(sigma) = (1/S_yc) ((m+1)/2) max_{i<j} (|s_i - s_j| + K (s_i + s_j)) - 1,
 *   K = (m-1)/(m+1), s_k the principal stresses (eigenvalues of sigma),
 *   m = S_yc / S_yt (S_yc, S_yt the uniaxial compressive and tensile yield
 *   stresses; f = 0 at uniaxial compression -S_yc and tension S_yt).
 * For m > 0 the maximising pair is always the extreme pair, so with ascending
 * eigenvalues f = (m lambda_3 - lambda_1) / S_yc - 1; the eigenvalues come
 * from Algorithm 6 on the stable invariants in the requested precision.
 * The gradient is the vector-Jacobian product of the eigenvalues with the
 * weights (-1/S_yc, 0, m/S_yc) (eig3_eigvals_backward's formula and layout
 * convention: for EIG3_SYM6 it is taken with respect to the six stored
 * entries, an off-diagonal entry receiving G_ij + G_ji).  Where two computed
 * eigenvalues coincide exactly their weights are replaced by their mean,
 * which gives the average of the one-sided gradients -- an element of the
 * subdifferential of this convex function of a symmetric sigma.  The
 * eigenvalues and the gradient are computed in one pass per matrix; nothing
 * but f and grad_sigma is written.
 *   sigma       device, n matrices (read only).
 *   s_yc, m     positive finite constants (otherwise EIG3_ERR_ARG).
 *   f           device, n values of `dtype`.
 *   grad_sigma  device, n x 9 or n x 6 of `dtype`, or NULL for the value only.
 */
eig3_status eig3_mohr_coulomb(const void *sigma, int layout, int dtype, int precision, int64_t n,
                              double s_yc, double m, void *f, void *grad_sigma, void *stream);

/*
 * eig3_eigvals_variant -- the invariant evaluations that Sections J2, J3,
 * Delta and Eigenvalues compare, each followed by Algorithm 6, in binary64
 * arithmetic, for measuring their stability on large batches.  Not the
 * method: use eig3_invariants / eig3_eigvals for results.
 *   variant  EIG3_VARIANT_PRESENT       Algorithms 1, 2, 4, 5 (the values of
 *                                       eig3_invariants and eig3_eigvals);
 *            EIG3_VARIANT_NAIVE         Algorithm 3 and the naive J3 monomial
 *                                       sum, Delta = 4 J2^3 - 27 J3^2;
 *            EIG3_VARIANT_NAIVE_TENSOR  S = A - tr(A)/3 I, J2 = tr(S S)/2,
 *                                       J3 = det S (first-row cofactor
 *                                       expansion), Delta = 4 J2^3 - 27 J3^2.
 *            Anything else: EIG3_ERR_ARG.
 *   The naive forms are evaluated as printed, every monomial and sum left
 *   to right with separately rounded binary64 operations (no FMA), and with
 *   no scaling, so they over/underflow where the printed formulas do.
 *   A        device, n matrices (read only); precision is binary64 for every
 *            dtype.
 *   inv      device, n x 4 binary64 (I1, J2, J3, Delta), or NULL.
 *   lam      device, n x 3 of `dtype` (ascending eigenvalues), or NULL.
 *            At least one of inv and lam is required (else EIG3_ERR_ARG).
 */
eig3_status eig3_eigvals_variant(const void *A, int layout, int dtype, int variant, int64_t n,
                                 double *inv, void *lam, void *stream);

/* Set a device eig3_stats to (0, 0, 0, +inf, 0, 0) on `stream`. */
eig3_status eig3_stats_reset(eig3_stats *stats, void *stream);

/* Human-readable name of a status code (static string). */
const char *eig3_status_string(int status);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int eig3_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EIG3_H */
