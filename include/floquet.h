/*
 * floquet.h -- C ABI of the GB300 geometric-sum polynomial-filter Floquet eigensolver.
 *
 * Method: D. J. Luitz, "Polynomial filter diagonalization of large Floquet unitary
 * operators", arXiv:2102.05054. The eigenpairs of a Floquet unitary U closest to a target
 * exp(i phi) on the unit circle are found by Arnoldi iteration (Sec. 4, Eq. arnoldi) on the
 * geometric-sum filter g_k(U) (Sec. 3, Eq. geo), followed by Rayleigh quotients
 * omega = <n|U|n> and residuals ||U|n> - omega|n>|| (Sec. 4, Eq. residual).
 *
 * Operator (a local Floquet operator with a cheap matrix-free product, as Sec. 2 requires):
 *   U = D K,  K = exp(-i g sum_i X_i),  D = exp(-i sum_i (J Z_i Z_{i+1} + h_i Z_i)),
 *   periodic chain of L qubits (bond (L-1, 0) included), 3 <= L <= 24.
 *   Amplitude index s = sum_i b_i 2^i (qubit i = bit i), Z|0> = +|0>.
 * The paper's own operator, a brickwork circuit of two-qubit gates (Sec. 2), is available
 * through brickwork_create; its handle works with the same calls (see there).
 *
 * Filter length: k is the NUMBER OF TERMS, g_k(U) = sum_{j=0}^{k-1} exp(-i j phi) U^j.
 * (The paper's order-k filter, Eq. geo, has k+1 terms.)
 *
 * Layout: a state is d = 2^L complex numbers, interleaved (re, im); complex128 = two
 * doubles, complex64 = two floats. A block of n states is column-major with leading
 * dimension d (state j starts at element j*d).
 *
 * Pointers: "device" pointers are CUDA device (or managed) memory of the current device;
 * "host" pointers are ordinary host memory. Arguments documented "host or device" are
 * classified with cudaPointerGetAttributes. The caller owns every buffer it passes; the
 * library owns the workspace it allocates inside a floquet_t (freed by floquet_destroy)
 * and the scratch of a call (freed before the call returns).
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream). Calls that return
 * host-visible results synchronise that stream before returning; the others are
 * asynchronous with respect to the host.
 *
 * Errors: every call returns FLOQUET_OK (0) or a negative code; floquet_last_error()
 * returns a thread-local message describing the last failure. No C++ exception crosses the
 * ABI. After FLOQUET_ECUDA the CUDA context may be unusable.
 */
#ifndef FLOQUET_H
#define FLOQUET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct floquet_op* floquet_t;

enum floquet_status {
  FLOQUET_OK = 0,
  FLOQUET_EINVAL = -1,   /* invalid argument (size, pointer, enum) */
  FLOQUET_ENOMEM = -2,   /* device or host allocation failed */
  FLOQUET_ECUDA = -3,    /* a CUDA call or kernel failed */
  FLOQUET_ENOCONV = -4,  /* eigensolver hit max_restarts; partial results returned */
  FLOQUET_ETIMEOUT = -5  /* reserved: a bounded device-side wait gave up */
};

/* Element types of states passed across the ABI, and the precision of the U sweeps:
 *   FLOQUET_C128    -- complex128 in and out, complex128 (FP64) sweeps;
 *   FLOQUET_C64     -- complex64 in and out, complex64 (FP32) sweeps;
 *   FLOQUET_C128_DF -- complex128 in and out, sweeps in double-float complex arithmetic
 *                      (each real an unevaluated sum of two floats, ~48 significant bits,
 *                      error-free transformations on the FP32 pipes). */
enum floquet_dtype { FLOQUET_C128 = 0, FLOQUET_C64 = 1, FLOQUET_C128_DF = 2 };

/* Precision form of the eigensolver (arnoldi_eigs):
 *   FLOQUET_FP64        -- filter sweeps U^j in complex128, FP64 Arnoldi;
 *   FLOQUET_FILTER_FP32 -- filter sweeps in complex64 with complex64 accumulation, FP64
 *                          Gram-Schmidt, Hessenberg/Schur, Ritz extraction and residuals,
 *                          then an FP64 Rayleigh-Ritz polish of the returned eigenpairs
 *                          (Sec. 4 footnote: one Ritz step with <n|U|m> on approximate
 *                          eigenvectors) iterated with defect-corrected filtering until the
 *                          U-residuals reach tol_resid. */
/*   FLOQUET_FILTER_DF   -- filter sweeps in double-float (FLOQUET_C128_DF), FP64 for the
 *                          rest; no polish needed (sweep accuracy ~1e-14 per step). */
enum floquet_precision { FLOQUET_FP64 = 0, FLOQUET_FILTER_FP32 = 1, FLOQUET_FILTER_DF = 2 };

/* Filter formulation (filter_apply): both equal sum_{j<k} z^j U^j psi, z = exp(-i phi).
 *   FLOQUET_FORM_ACC    -- psi_0 = psi, psi_{j+1} = U psi_j, acc += z^j psi_j: 4 d b bytes
 *                          per U application (b = bytes per complex);
 *   FLOQUET_FORM_HORNER -- acc <- psi + z U acc, k-1 times from acc = psi: 3 d b bytes
 *                          per U application. */
enum floquet_form { FLOQUET_FORM_ACC = 0, FLOQUET_FORM_HORNER = 1 };

/* Create the paper's own Floquet operator instead (Sec. 2, Eqs. U, unitary): a two-layer
 * brickwork circuit on L qubits (L even, 4 <= L <= 24), U = U_a U_b with
 *     U_b = u_0 u_{1,2} u_{3,4} ... u_{L-3,L-2} u_{L-1}   (acts first),
 *     U_a = u_{0,1} u_{2,3} ... u_{L-2,L-1},
 * qubit i = bit i of the amplitude index. g2: host, (L-1) bond gates u_{i,i+1}, each a
 * row-major 4 x 4 complex matrix (interleaved re, im: element (r, c) of bond i at doubles
 * 32 i + 2 (4 r + c)) whose indices are b_i + 2 b_{i+1}; g1: host, u_0 then u_{L-1}, row-major
 * 2 x 2 complex (16 doubles). Gates are copied and are expected to be unitary (the paper
 * draws them from the Haar measure). The matrix-free product is the paper's Eq. matvec: U is
 * split at an odd qubit q into U_L (qubits 0..q) and U_R (qubits q..L-1), U = (U_L x 1)
 * (1 x U_R), both built here as dense float64 matrices of side 2^(q+1) and 2^(L-q), and
 * every U application is two complex GEMMs on two reshapes of the state (cuBLAS ZGEMM for
 * complex128; for FLOQUET_C128_DF this library's split-K double-float GEMM on the FP32
 * pipes). The returned handle works with floquet_apply_u (complex128), filter_apply
 * (complex128 in both forms, double-float in the Horner form), ritz_residuals and
 * arnoldi_eigs (FLOQUET_FP64 or FLOQUET_FILTER_DF); other dtypes, forms and precisions give
 * FLOQUET_EINVAL. Allocates U_L, U_R (float64 and double-float) and a 32 MiB cuBLAS
 * workspace on the current device. */
int brickwork_create(int L, const double* g2, const double* g1, floquet_t* out);

/* Create the operator U = D K (Sec. 2; model fixed above). h: host, L doubles, copied.
 * Builds the diagonal-phase tables and the pass plan on the current device.
 * EINVAL if L outside [3, 24] or h/out NULL; ENOMEM/ECUDA on allocation failure. */
int floquet_create(int L, double J, double g, const double* h, floquet_t* out);

/* Release the operator and all workspace it owns. NULL is accepted. */
int floquet_destroy(floquet_t op);

/* d = 2^L. */
int floquet_dim(floquet_t op, int64_t* d);

/* psi_out[:, j] = U psi_in[:, j] for j < nvec (the matrix-free product of Sec. 2 that
 * Sec. 3 requires). psi_in, psi_out: device, nvec*d complex of `dtype`; may be equal
 * (in place). Asynchronous on `stream`. */
int floquet_apply_u(floquet_t op, const void* psi_in, void* psi_out, int nvec, int dtype,
                    void* stream);

/* psi_out[:, j] = g_k(U) psi_in[:, j] (Sec. 3, Eq. geo, k terms) for j < nvec.
 * psi_in, psi_out: device, nvec*d complex of `dtype`, must not overlap. k >= 1.
 * `form` selects the formulation (floquet_form). Asynchronous on `stream`; the k-step loop
 * runs as a captured CUDA graph that is cached in `op` for the same (k, nvec, dtype, form). */
int filter_apply(floquet_t op, double phi, int64_t k, const void* psi_in, void* psi_out,
                 int nvec, int dtype, int form, void* stream);

/* The correction step of the FP64 polish of the FP32-filter form (Sec. 4 footnote, iterated),
 * exposed for testing and for callers that refine eigenpairs themselves. For each j < n:
 *     out_j = q_j(U) r_j,   q_j(U) = sum_{l=0}^{K-2} a_l U^l,
 *     a_l = z^{l+1} g_{K-1-l}(z omega_j),  z = exp(-i phi),  g_n(w) = sum_{m<n} w^m,
 * the polynomial with g_K(U) - g_K(omega_j) = q_j(U) (U - omega_j) (Sec. 3, Eq. geo, summed
 * term by term). For r_j = (U - omega_j) x_j this is g_K(U) x_j - g_K(omega_j) x_j: the
 * filtered vector formed from the small residual only, so the sweeps' rounding is relative to
 * ||r_j||. The coefficients are formed in float64 on the host and rounded to the sweep
 * precision.
 *   phi   -- filter target; K >= 2 filter length;
 *   omega -- host, 2n doubles (re, im), any finite values;
 *   R     -- device, d x n complex128 (r_j at R + j d); out: device, d x n complex128, must not
 *            overlap R;
 *   sweep -- FLOQUET_C64 (complex64 sweeps) or FLOQUET_C128_DF (double-float sweeps).
 * Allocates and frees small scratch; synchronises `stream`. EINVAL for a NULL pointer, n < 1,
 * K < 2, another sweep type, phi or omega not finite, overlapping R and out, or a brickwork
 * handle. */
int floquet_polish_correction(floquet_t op, double phi, int64_t K, const double* omega,
                              const void* R, void* out, int n, int sweep, void* stream);

/* Host-only query of the U application's pass plan (no GPU needed): the passes that split
 * the L qubits' X kicks (Sec. 2, matrix-free product) for tiles of 2^NB amplitudes whose later
 * passes keep at least min_cols contiguous low bits. For pass i, out[6i .. 6i+5] =
 * (NB, c, start, kick_from, midbits, topshift): the tile holds global bits [0, c) and
 * [start, start + NB - c), the pass kicks tile bits [kick_from, NB), and the kernels place
 * tile bits at c.. with the shifts midbits = start - c and topshift = start + NB - c (0 and L
 * for a single pass). *n_passes receives the count; EINVAL for L outside [1, 30], NB < 1,
 * min_cols outside [0, NB), NULL pointers or fewer than *n_passes slots. */
int floquet_pass_plan(int L, int NB, int min_cols, int* out, int max_passes, int* n_passes);

/* One classical Gram-Schmidt step with one full reorthogonalisation (CGS2) of Sec. 4's
 * Arnoldi process: w <- (w - V V^H w) / beta, twice projected, for n >= 0 orthonormal
 * columns V (device, d x n complex128, column-major, leading dimension d).
 * w: device, d complex128, overwritten with the unit vector. h: host, n+1 complex128
 * (2(n+1) doubles): the summed projection coefficients V^H w and, last, beta (real part).
 * Synchronises `stream`. */
int gram_schmidt(int64_t d, const void* V, int n, void* w, double* h, void* stream);

/* The CGS2 step of gram_schmidt for callers that cannot allocate device memory while they
 * run (a process that reserves its whole memory budget at start-up, or a latency-critical
 * loop that cannot afford the device-wide synchronisation cudaFree implies). The paper has no
 * counterpart: this is a deployment variant of gram_schmidt. It calls no allocator: its
 * scratch is a fixed file-scope device array of 2.1 MiB that every GPU loading the library
 * holds until exit; the caller passes all inputs and outputs.
 *   d    -- rows, 1 <= d <= 2^20 (larger: FLOQUET_EINVAL, nothing launched);
 *   V    -- device, d x n complex128, orthonormal columns, leading dimension d;
 *   n    -- columns, 0 <= n <= 256 (larger: FLOQUET_EINVAL);
 *   w    -- device, d complex128, overwritten with the unit vector;
 *   h    -- device, n+1 complex128 (caller-owned): the summed coefficients V^H w, then beta.
 * Asynchronous on `stream`. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any stream
 * capture. All calls share the one array and it keeps the last call's contents (nothing in
 * it needs to start at zero): calls that overlap on the GPU race and must be serialised by
 * the caller. */
int gram_schmidt_noalloc(int64_t d, const void* V, int n, void* w, void* h, void* stream);

/* Eigen-decomposition of a small general complex matrix on the device (the Hessenberg /
 * Schur solve behind Sec. 4's Ritz pairs): A = Y diag(lambda) Y^{-1}.
 * A: host or device, n x n complex128 column-major; lambda: host, n complex128; Y: host or
 * device, n x n complex128 column-major, unit-norm columns. 1 <= n <= 512. Order of the
 * eigenvalues: descending modulus. Synchronises `stream`. */
int small_eig(int n, const void* A, double* lambda, void* Y, void* stream);

/* Rayleigh quotients and residuals (Sec. 4, Eq. residual) of nvec vectors X (device, d x
 * nvec complex128; normalised internally, X itself is not modified):
 * omega_j = <x_j|U|x_j>/<x_j|x_j>, resid_j = ||U x_j - omega_j x_j|| / ||x_j||.
 * omega: host, 2*nvec doubles; resid: host, nvec doubles. Synchronises `stream`. */
int ritz_residuals(floquet_t op, const void* X, int nvec, double* omega, double* resid,
                   void* stream);

/* The eigensolver of Secs. 3-4: Krylov-Schur restarted Arnoldi on g_k(U) with CGS2,
 * Krylov dimension m, keeping the nev eigenpairs of U whose eigenvalues are closest to
 * exp(i phi) by wrapped angle |arg(omega e^{-i phi})| (ties: ascending arg), eigenvalues as
 * Rayleigh quotients and residuals as in Eq. residual.
 *   precision   -- floquet_precision;
 *   tol         -- convergence tolerance of the Ritz values of g_k(U) relative to |theta|
 *                  (<= 0: 1e-12 for FP64, 1e-7 for FILTER_FP32);
 *   tol_resid   -- required U-residual of every returned pair (<= 0: 1e-10);
 *   max_restarts-- restart limit (ENOCONV when reached, partial results returned);
 *   v0          -- host or device, d complex128 start vector (need not be normalised).
 * Outputs: evals host 2*nev doubles (re, im), sorted by closeness; evecs host or device
 * d*nev complex128 (may be NULL); resid host nev doubles; n_conv host int: number of
 * returned pairs meeting tol_resid. A pair the solver did not find (FLOQUET_ENOCONV, e.g.
 * a start vector inside an invariant subspace smaller than nev) is returned as eigenvalue 0
 * with residual +infinity. 1 <= nev < m <= min(d, 512), 2 <= k <= 2^24.
 * Synchronises `stream`. */
int arnoldi_eigs(floquet_t op, double phi, int64_t k, int nev, int m, int precision,
                 double tol, double tol_resid, int max_restarts, const void* v0,
                 double* evals, void* evecs, double* resid, int* n_conv, void* stream);

/* Many independent eigenproblems in lockstep on one GPU: R disorder realisations (h: host,
 * R*L doubles, realisation r at h + r*L) times P targets (phis: host, P doubles), all with
 * the same L, J, g, k, nev, m. Problem q = r*P + p. precision: FLOQUET_FP64 or
 * FLOQUET_FILTER_DF (double-float sweeps; FLOQUET_FILTER_FP32 is not offered for batches:
 * FLOQUET_EINVAL). v0: host or device, d complex128, shared start vector. Outputs (host):
 * evals 2*nev*R*P doubles, resid nev*R*P, n_conv R*P; problem q's block starts at q*nev.
 * Synchronises `stream`. */
int arnoldi_eigs_batched(int L, double J, double g, const double* h, int R,
                         const double* phis, int P, int64_t k, int nev, int m, int precision,
                         double tol, double tol_resid, int max_restarts, const void* v0,
                         double* evals, double* resid, int* n_conv, void* stream);

/* The paper's choice of filter length and Krylov dimension (Sec. 4, strategy paragraph;
 * Sec. 5, parameter scan of Fig. bench): the runtime is minimal when the Krylov dimension is
 * about 80 % of the number of eigenvalues on the outer lobe of g_k (2d/k with k terms), and
 * for large
 * sizes the paper takes n_cv = floor(2^(L/2 + 1)) with k = 0.8 * 2^(L+1) / n_cv, and
 * n_cv > 2 nev. This library computes
 *     m = max(floor(2^(L/2 + 1)), 2 nev + 1), capped at min(max_m, d - 1),
 *     k = round(2^(L+3) / (5 m))   (= 0.8 * 2^(L+1) / m, never a tie), at least 2,
 * in integer arithmetic (floor(2^(L/2+1)) is the integer square root of 2^(L+2)). The
 * paper does not say how k is rounded; capping m (the small eigensolver takes m <= 512)
 * keeps the m k ~ 0.8 * 2d relation by recomputing k from the capped m.
 * Host only (no GPU needed). 3 <= L <= 24, nev >= 1, 2 nev + 1 <= min(max_m, d - 1);
 * otherwise FLOQUET_EINVAL. k and m are host pointers. */
int floquet_suggest_params(int L, int nev, int max_m, int64_t* k, int* m);

/* Entanglement entropy of states (Sec. 5, Eq. ee): for each state j and cut c, subsystem A =
 * qubits 0 .. cuts[c] - 1 (the low bits of the amplitude index), B = the rest, and
 *     S[j * ncut + c] = -sum_i lambda_i ln lambda_i
 * over the eigenvalues lambda_i of the reduced density matrix of A (the squared singular
 * values of the state as a 2^{L_A} x 2^{L - L_A} matrix). Computed on the GPU in float64:
 * the Gram matrix of the smaller side, Householder tridiagonalisation, bisection. The paper's
 * chain has open boundaries and one cut; this library's chain is periodic, so a block of
 * L_A qubits has two boundaries, and the formula is the same.
 * X: device, nvec states of d = 2^L complex128 (state j at X + j d), assumed normalised.
 * cuts: host, ncut values in [0, L] (0 and L give 0). S: host, nvec * ncut doubles.
 * Allocates device workspace (at most ~4 GiB per cut, processed in chunks of states).
 * Synchronises `stream`. 1 <= L <= 24, 1 <= nvec <= 65535, min(L_A, L - L_A) <= 11 (the
 * Householder reduction runs in one CTA per matrix of side 2^min(L_A, L - L_A)). */
int entanglement_entropy(int L, const void* X, int nvec, const int* cuts, int ncut, double* S,
                         void* stream);

/* Measurement hook. While enabled (on != 0), every replay of a filter's k-step sweep graph is
 * bracketed by CUDA events on the stream it runs on, and the library accumulates the
 * elapsed device time, the number of U applications (vectors x steps) and their
 * algorithmic bytes (4 d b per U application in the accumulate form, 3 d b in the Horner
 * form; b = 16 for complex128, 8 for complex64), separately for complex64 (index 1) and
 * complex128 (index 0) sweeps, double-float sweeps at index 2 (b = 16).
 * floquet_profile_read synchronises the event pairs it reads and returns the totals since
 * the last floquet_profile_enable(1); arrays of length 3. */
int floquet_profile_enable(int on);
int floquet_profile_read(double* sweep_ms, int64_t* u_applications, double* alg_bytes);

/* Number of kernel launches issued by this library on the calling thread since the last
 * call of floquet_reset_launch_count (graph replays count each kernel node). */
int64_t floquet_launch_count(void);
void floquet_reset_launch_count(void);

/* Thread-local description of the last error ("" if none). Valid until the next call. */
const char* floquet_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLOQUET_H */
