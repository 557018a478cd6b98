/*
 * dacp.h -- C ABI of the GB300 implementation of DACP ("dual application of
 * Chebyshev polynomial", Guan & Zhang, arXiv 2011.02107): thousands of central
 * eigenvalues of spin-1/2 Hamiltonians
 *
 *     H = sum_{i<j} J_ij Z_i Z_j + sum_i h_i Z_i + sum_i Gamma_i X_i
 *
 * on 2^N-dimensional real state vectors, matrix-free (Sec. II intro; the
 * paper's sigma^x sigma^x + sigma^z models of Sec. III are this form after a
 * global Hadamard rotation). Z_i acts on bit i of the basis-state index.
 * dacp_set_pair_couplings adds sum_{i<j} (Jxx_ij X_i X_j + Jyy_ij Y_i Y_j)
 * (XXZ and Heisenberg chains; the vectors stay real).
 *
 * Conventions for every entry point
 *   - Return a dacp_status; nothing throws across the ABI. On failure the
 *     handle keeps a message readable with dacp_last_error().
 *   - All host arrays are owned by the caller and only read or written during
 *     the call. The library owns every device buffer it allocates.
 *   - Work is ordered on the handle's CUDA stream: the `stream` given to
 *     dacp_create, or a private non-blocking stream when it is NULL. Every
 *     call has finished its device work when it returns.
 *   - A handle is not thread-safe; separate handles are independent.
 *   - Calling out of order (e.g. dacp_central_eigs before dacp_basis_moments)
 *     returns DACP_ERR_STATE.
 *   - Per-realization failures inside a batch are reported through n_found[r]
 *     = -status, so one bad realization does not fail the batch.
 */
#ifndef DACP_H
#define DACP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dacp_ctx* dacp_handle;

typedef enum {
    DACP_OK = 0,
    DACP_ERR_ARG = 1,          /* bad argument (sizes, NULL, range)            */
    DACP_ERR_CUDA = 2,         /* CUDA runtime error                            */
    DACP_ERR_NOMEM = 3,        /* device allocation failed                      */
    DACP_ERR_NUMERIC = 4,      /* NaN/Inf, or E_max is not a bound (|mu_k|>mu_0)*/
    DACP_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                 */
    DACP_ERR_STATE = 6,        /* call out of order                             */
    DACP_ERR_NOT_CONVERGED = 7,/* eigensolver reported failure                  */
    DACP_ERR_LIBRARY = 8       /* cuSOLVER / cuBLAS error                       */
} dacp_status;

typedef enum {
    DACP_FP64 = 0,             /* float64 vectors, float64 moments (plain DACP) */
    DACP_FP32 = 1,             /* float32 vectors, float64 moments and solve    */
    DACP_DF32 = 2              /* double-float vectors (pairs of float32, about
                                  48 significant bits, float32 arithmetic with
                                  error-free transformations), float64 moments
                                  and solve                                     */
} dacp_precision;

/*
 * dacp_create -- build a batch of n_real independent problems ("realizations").
 *
 *   n_spins[r]   N_r, 1 <= N_r <= 26.
 *   J            concatenated row-major N_r x N_r zz couplings; only i<j read.
 *                Realization r starts at sum_{r'<r} N_r'^2.
 *   h, gamma     concatenated z-fields and x-fields, N_r each.
 *   block_b      start vectors per realization (block filter, Sec. III):
 *                1, 2 or 4.
 *   precision    dacp_precision.
 *   psi0         start vectors, float64, realization r at sum_{r'<r} 2^N_r' * b,
 *                layout [state][column]. The paper draws them at random
 *                (Sec. II intro); the caller supplies them.
 *   stream       cudaStream_t or NULL.
 * Errors: DACP_ERR_ARG for bad sizes, DACP_ERR_NOMEM if device memory runs out
 * (nothing is leaked; *out stays NULL).
 */
dacp_status dacp_create(dacp_handle* out, int n_real, const int* n_spins,
                        const double* J, const double* h, const double* gamma,
                        int block_b, int precision, const double* psi0, void* stream);

/*
 * dacp_set_pair_couplings -- add two-body flip couplings
 *   sum_{i<j} (Jxx_ij X_i X_j + Jyy_ij Y_i Y_j)
 * to every realization's H. These give XXZ and Heisenberg chains, and the
 * paper's own sigma^x sigma^x couplings (Sec. III) without the Hadamard
 * rotation. Both terms flip bits i and j. Y_i Y_j carries the real sign
 * -z_i(s) z_j(s), so the vectors stay real.
 *   Jxx, Jyy  concatenated row-major N_r x N_r blocks laid out like J in
 *             dacp_create (only i<j read). NULL means all zero. Copied; the
 *             caller keeps ownership.
 * A call replaces the couplings of any earlier call; all zero removes them.
 * The Pauli 1-norm that clamps the E_max bound grows by sum |Jxx| + |Jyy|.
 * Every stencil pass (filter, evolution, Lanczos, KPM, dacp_apply_h) then
 * includes the pair flips, read element by element. The launch uses the
 * generic kernels rather than the ones specialised on a uniform tile size.
 * Parameters and results are reset (as after dacp_create): set or choose
 * parameters again.
 * Errors: DACP_ERR_ARG for a non-finite coupling; DACP_ERR_NOMEM, DACP_ERR_CUDA.
 */
dacp_status dacp_set_pair_couplings(dacp_handle hd, const double* Jxx, const double* Jyy);

/*
 * dacp_set_global_flips -- add c_r X_0 X_1 ... X_{N_r - 1} (every spin of the
 * realization flipped at once) to realization r's H. It is the term that the
 * parity-sector reduction below leaves in each sector, and a model term in its
 * own right.
 *   coef  n_real doubles (copied; the caller keeps ownership), NULL or all
 *         zero removes the term.
 * Every stencil pass reads the partner s XOR (2^N - 1) (global memory, or the
 * tile when the realization is one tile). The Pauli 1-norm that clamps the
 * E_max bound grows by |c_r|. Parameters and results are reset (as after
 * dacp_create). Errors: DACP_ERR_ARG for a non-finite coefficient;
 * DACP_ERR_NOMEM, DACP_ERR_CUDA.
 */
dacp_status dacp_set_global_flips(dacp_handle hd, const double* coef);

/*
 * dacp_create_parity_sectors -- a handle whose realizations are the two parity
 * sectors of each input realization. The paper's models without z-fields
 * (Sec. III; the spin-glass shards) commute with P = X_0 X_1 ... X_{N-1}, so H
 * splits into the sectors P = +1 and -1 of 2^(N-1) states each, whose levels
 * together are H's levels. In the basis (|s> + sigma |s XOR (2^N - 1)>) / sqrt 2
 * (s with bit N-1 clear) sector sigma is the (N-1)-spin model
 *     sum_{i<j<N-1} J_ij Z_i Z_j + sum_{i<N-1} J_{i,N-1} Z_i
 *       + sum_{i<N-1} Gamma_i X_i + sigma Gamma_{N-1} X_0 ... X_{N-2}
 * (z-fields from the couplings to spin N-1, a global flip from its x-field).
 * Each sector holds half the levels at half the density: for the same number
 * of central levels a sector needs half the evolution orders on half-size
 * vectors and a basis of half the size.
 *   n_real, n_spins (2 .. 26), J, gamma, block_b, precision, stream: as
 *            dacp_create for the full models; h must be all zero
 *            (DACP_ERR_ARG otherwise).
 *   psi0     start vectors of the 2 n_real sector realizations: realization
 *            2r is sector +1 of input r, 2r+1 sector -1, each 2^(N_r - 1) x b
 *            float64, [state][column], concatenated in that order.
 * The result is an ordinary handle of 2 n_real realizations of N_r - 1 spins;
 * dacp_merge_sectors turns their levels back into the inputs' levels.
 */
dacp_status dacp_create_parity_sectors(dacp_handle* out, int n_real, const int* n_spins, const double* J,
                                       const double* h, const double* gamma, int block_b, int precision,
                                       const double* psi0, void* stream);

/*
 * dacp_merge_sectors -- host arithmetic only: the levels of n_real
 * realizations from those of their two sectors (realizations 2r and 2r+1 of a
 * dacp_create_parity_sectors handle). Each sector returned the levels of
 * smallest |E| it has, so the union holds every level up to the smaller of
 * the two sectors' largest |E|; of those, the n_eigs of smallest |E| come back,
 * ascending.
 *   eigs_in, n_found_in  the sectors' results, [2 n_real][n_in] and [2 n_real],
 *                        as dacp_central_eigs / dacp_solve write them.
 *   eigs, n_found        [n_real][n_eigs] and [n_real]: n_found[r] < n_eigs
 *                        when the union cannot vouch for n_eigs levels (ask the
 *                        sectors for more); a failed sector's -status passes on.
 * Errors: DACP_ERR_ARG for bad sizes or NULL.
 */
dacp_status dacp_merge_sectors(int n_real, int n_in, const double* eigs_in, const int* n_found_in, int n_eigs,
                               double* eigs, int* n_found);


/*
 * dacp_set_params -- explicit per-realization parameters (arrays of n_real).
 *   emax  bound on |E| (E_min = -E_max, Sec. II A); must be a true bound.
 *   a     window half-width, 0 < a < emax (Sec. II A).
 *   K     filter order (Eq. target; the paper uses K = 18 E_max / a). K >= 0.
 *   n     basis half-size: b(2n+1) basis vectors (Eq. set / set2). n >= 1.
 * Resets any filter or moment results. Errors: DACP_ERR_ARG.
 */
dacp_status dacp_set_params(dacp_handle hd, const double* emax, const double* a,
                            const int* K, const int* n);

/*
 * dacp_choose_params -- the parameter heuristic of Sec. III on the GPU:
 *   E_max: Lanczos upper-bound estimator (lanczos_steps steps on column 0 of
 *          psi0, bound = max|Ritz| + residual norm, x(1+1e-3), clamped to the
 *          Pauli 1-norm);
 *   a:     kernel-polynomial DOS estimate from kpm_moments Chebyshev moments of
 *          the same vector; [-a, a] holds d = d_ratio * n_eigs levels;
 *   n:     b(2n+1) >= basis_ratio * d (Sec. II B: 2n+1 = 1.5 d);
 *   K:     ceil(c_order * E_max / a) (Sec. II A: c_order = 18). c_order <= 0
 *          picks the precision default: 18 for DACP_FP64 and DACP_DF32, 6 for DACP_FP32
 *          (float32 moments resolve a dynamic range of about e^12).
 * Errors: DACP_ERR_ARG, DACP_ERR_CUDA.
 */
dacp_status dacp_choose_params(dacp_handle hd, int n_eigs, double d_ratio,
                               double basis_ratio, double c_order,
                               int lanczos_steps, int kpm_moments);

/* dacp_get_params -- copy the parameters in use (each pointer may be NULL);
 * kn[r] = k_n = floor(n pi / a_r), the last basis order (Eq. set2). */
dacp_status dacp_get_params(dacp_handle hd, double* emax, double* a, int* K,
                            int* n, int* kn);

/*
 * dacp_filter -- the exp-semicircle filter (Sec. II A, Eqs. F, chevo, target):
 * psi_E = T_K(F) psi0 / norm, F = (H^2 - E_c)/E_0, per column, by the
 * three-term recurrence (two fused H.v sweeps per order). Requires params.
 */
dacp_status dacp_filter(dacp_handle hd);

/*
 * dacp_basis_moments -- the Chebyshev evolution (Sec. II B, Appendix C):
 * w_{k+1} = 2 G w_k - w_{k-1}, G = H/E_max, w_0 = psi_E, for k = 0..k_n,
 * accumulating the float64 moment blocks
 *   mu_j^{pq} = <psi_E^p| T_j(G) |psi_E^q>,  j = 0 .. 2 k_n + 1,
 * through T_2k = 2 T_k^2 - 1 and T_{2k+1} = 2 T_{k+1} T_k - T_1. The basis
 * vectors themselves are never stored (Appendix C). Requires dacp_filter.
 * Errors: DACP_ERR_NUMERIC when a realization's |mu_j| exceeds mu_0 (E_max
 * was not a bound) -- reported per realization by dacp_central_eigs.
 */
dacp_status dacp_basis_moments(dacp_handle hd);

/*
 * dacp_central_eigs -- assemble S and H from the moments (Appendix C,
 * S_ij = (mu_{x_i+x_j} + mu_{|x_i-x_j|})/2 and the same with
 * nu_k = E_max (mu_{k+1} + mu_{|k-1|})/2 for H), solve H B = S B Lambda
 * (Eq. gep) after dropping eigenvalues of S below eps * lambda_max(S)
 * (eps <= 0 -> 1e-12 for DACP_FP64 as in Sec. II C, 1e-6 for DACP_FP32,
 * whose moments carry float32 round-off, 1e-11 for DACP_DF32), and return up to n_eigs eigenvalues of
 * smallest |E| inside [-window, window] (window <= 0 -> a) in ascending order.
 *   eigs     n_real * n_eigs doubles; realization r at r * n_eigs.
 *   n_found  n_real ints: count written for r, or -dacp_status on failure.
 *   rank     n_real ints (may be NULL): m, the retained rank of S.
 */
dacp_status dacp_central_eigs(dacp_handle hd, int n_eigs, double window, double eps,
                              double* eigs, int* n_found, int* rank);

/*
 * dacp_solve -- dacp_filter, dacp_basis_moments and dacp_central_eigs in one
 * call, with the subspace solves overlapped with the evolution: realizations
 * finish their evolution at different orders (k_n differs), and each group of
 * finished realizations is solved (batched cuSOLVER / cuBLAS on a second
 * stream, driven by a worker thread) while the rest keep evolving. Results
 * are those of the three separate calls up to the rounding of the batched
 * eigensolver (the batch composition sets the padded size).
 * Arguments and per-realization failures as in dacp_central_eigs. Requires
 * parameters; leaves the handle as dacp_basis_moments does (moments kept for
 * dacp_get_moments / dacp_residuals). dacp_get_timings then gives T_F, T_E and
 * the part of the subspace solves that ran after the evolution ended.
 */
dacp_status dacp_solve(dacp_handle hd, int n_eigs, double window, double eps, double* eigs, int* n_found,
                       int* rank);

/*
 * dacp_get_moments -- copy realization r's moments mu[j][p][q], j = 0..2k_n+1
 * (float64, (2 k_n + 2) b^2 values) into mu (capacity cap doubles).
 * *count receives the number of doubles. Test hook.
 */
dacp_status dacp_get_moments(dacp_handle hd, int r, double* mu, int64_t cap, int64_t* count);

/*
 * dacp_residuals -- the central levels of realization r together with their
 * residual norms ||r_j|| = sqrt(<H^2> - <H>^2) (Sec. II C), computed from the
 * moments alone: <H^2> of the Ritz vector phi_j = sum b_j[i,p] T_{x_i}(G) psi_p
 * is b_j^T H2 b_j, where H2_ij = (omega_{x_i+x_j} + omega_{|x_i-x_j|}) / 2 and
 * omega_k = <psi|H^2 T_k(G)|psi> = E_max^2 (mu_{k+2} + mu_k + mu_{|k-1|+1}
 * + mu_{||k-1|-1|}) / 4 (so the evolution runs one order beyond 2k_n+1).
 * ||r_j|| bounds the distance from the eigenvalue to the exact spectrum; the
 * moment form loses accuracy below about 1e-7 E_max (the difference of two
 * O(lam^2 + r^2) numbers), where it is clamped at 0.
 *   r        realization index.
 *   n_eigs, window, eps  as in dacp_central_eigs (same selection, same values).
 *   eigs, resid  host arrays of n_eigs doubles, written ascending in eigs.
 *   n_found  count written, or -dacp_status (DACP_ERR_NUMERIC,
 *            DACP_ERR_NOT_CONVERGED) when this realization failed.
 * Needs dacp_basis_moments first (else DACP_ERR_STATE). Allocates its own
 * workspace (O(M^2) doubles, M the basis size) and frees it before returning.
 */
dacp_status dacp_residuals(dacp_handle hd, int r, int n_eigs, double window, double eps, double* eigs,
                           double* resid, int* n_found);

/*
 * dacp_eigenvectors -- the central levels of realization r and their Ritz
 * vectors phi_j = sum_(i,p) b_j[i,p] T_{x_i}(G) psi_p (Appendix C: the
 * eigenvectors of H B = S B Lambda mapped back to the Hilbert space), the
 * eigenvector half of the error check of Sec. II C. The evolution of r is
 * replayed on the GPU and the 2n+1 basis orders T_{x_i}(G) psi_E are kept
 * as one float64 matrix V (2^N x b(2n+1)); Phi = V B_sel is one dgemm.
 *   r, n_eigs, window, eps  as in dacp_residuals (same selection).
 *   eigs     host array of n_eigs doubles (ascending).
 *   phi_dev  device array, column-major 2^N x n_found float64 with leading
 *            dimension ld >= 2^N, 8-byte aligned; column j is phi_j, with
 *            b_j^T S b_j = 1, i.e. unit norm up to rounding. Caller-owned.
 *   n_found  count written, or -dacp_status for a failed realization.
 * Workspace: V (8 * 2^N * b(2n+1) bytes) plus O(M^2), allocated and freed
 * here. Needs dacp_basis_moments first (else DACP_ERR_STATE).
 */
dacp_status dacp_eigenvectors(dacp_handle hd, int r, int n_eigs, double window, double eps, double* eigs,
                              double* phi_dev, int64_t ld, int* n_found);

/*
 * dacp_lanczos_filtered -- the comparison method of Appendix D on this
 * library's kernels: the exp-semicircle filter combined with the Lanczos
 * method. For realization r, with this handle's E_max, a and K: v_0 = column 0
 * of its start vectors, normalised; v_{j+1} = the part of T_K(F) v_j
 * (F = (H^2 - E_c)/E_0, one filter run of 2K H.v, Sec. II A) orthogonal to
 * v_0 .. v_j (classical Gram-Schmidt twice, float64), normalised, until
 * `steps` directions or a direction below 1e-8 of the filtered vector (1e-4
 * for DACP_FP32: the filter's own rounding); then Rayleigh-Ritz of H in the
 * space (V^T H V), the residual norms |H y - theta y| of its Ritz vectors,
 * and of the Ritz values with residual <= res_tol * E_max (res_tol <= 0 ->
 * 1e-8) the n_eigs of smallest |E| inside [-a, a], ascending.
 * T_K(F) is even in E, so the space does not separate levels E and -E: the
 * appendix's point that DACP is the more reliable route.
 *   steps     Krylov dimension, 1 .. min(4096, 2^N_r).
 *   eigs      host, n_eigs doubles; n_found the count written.
 *   dim       may be NULL: the dimension reached.
 *   ms        may be NULL, else 3 doubles: milliseconds of the filter runs,
 *             of the reorthogonalisation, of the Rayleigh-Ritz step.
 *   hv        may be NULL: H.v applied ((dim - 1) 2K + dim).
 * Memory: four float64 D x steps matrices plus O(steps^2), allocated and freed
 * here; the filter runs on a single-column handle of its own, on the same
 * stream. Needs parameters (else DACP_ERR_STATE); DACP_ERR_ARG for a bad r,
 * steps or n_eigs.
 */
dacp_status dacp_lanczos_filtered(dacp_handle hd, int r, int steps, int n_eigs, double res_tol, double* eigs,
                                  int* n_found, int* dim, double* ms, int64_t* hv);

/* dacp_get_filtered -- copy realization r's psi_E (2^N_r x b, float64) into
 * psi (capacity cap doubles). Test hook. */
dacp_status dacp_get_filtered(dacp_handle hd, int r, double* psi, int64_t cap);

/*
 * dacp_apply_h -- one matrix-free H.v of realization r (Sec. II intro):
 * y = H x for the b columns of x. x_dev, y_dev: device pointers to 2^N_r * b
 * values of the handle's precision, layout [state][column], 16-byte aligned,
 * not overlapping. Test hook. Values are float64 or float32 as they are; a
 * double-float value is the pair (hi, lo) of float32 with value hi + lo, and
 * with b = 4 each state's 32 bytes hold (hi_0, hi_1, lo_0, lo_1, hi_2, hi_3,
 * lo_2, lo_3) (the paired-float32 layout of the stencil), with b = 1 or 2
 * (hi, lo) per column.
 */
dacp_status dacp_apply_h(dacp_handle hd, int r, const void* x_dev, void* y_dev);

/*
 * dacp_get_timings -- milliseconds of the last filter, evolution and subspace
 * solve (T_F, T_E, T_D of Sec. III, Fig. 4), measured with CUDA events on the
 * handle's stream: ms[0] = T_F, ms[1] = T_E, ms[2] = T_D.
 */
dacp_status dacp_get_timings(dacp_handle hd, double* ms);

/*
 * dacp_autotune -- pick how the recurrences are launched by timing `orders`
 * evolution orders of this handle's own realizations for every candidate:
 * tile size (8 to 128 KB of the vector per CTA) x launch mode (per-order
 * launches replayed from a CUDA graph, one persistent cooperative launch
 * with a grid barrier per order, or -- float32 vectors, where the staged
 * tiles fit shared memory -- graph-replayed launches with staged tiles, mode 2
 * of dacp_set_launch). The fastest is kept and cached for the
 * process, keyed by (sorted N list, b, precision). Needs parameters; resets
 * filter and moment results (run dacp_filter again). *tile_bytes_out may be
 * NULL.
 */
dacp_status dacp_autotune(dacp_handle hd, int orders, int* tile_bytes_out);

/*
 * dacp_set_launch / dacp_get_launch -- set or read the launch mode (0 = graph
 * replay of per-order launches, 1 = persistent cooperative launch, 2 = as 0
 * with every HBM read of a tile -- the vector tile H acts on, the recurrence's
 * previous vectors and the diagonal -- staged in shared memory by bulk copies
 * at the start of the CTA; float32 vectors only) and tile size in bytes (power
 * of two, 1 KB to 128 KB). Mode 2 needs (1 + recurrence terms) tiles plus the
 * tile's diagonal in shared memory, so tiles above 64 KB are refused there
 * (DACP_ERR_ARG), as is mode 2 on float64 or double-float vectors. Setting
 * resets filter and moment results.
 */
dacp_status dacp_set_launch(dacp_handle hd, int mode, int tile_bytes);
dacp_status dacp_get_launch(dacp_handle hd, int* mode, int* tile_bytes);

/*
 * dacp_set_emax_rule -- how dacp_choose_params / dacp_choose_params_mlp turn
 * their k Lanczos steps into the bound E_max on |E| (Sec. III cites the
 * Lanczos upper-bound estimator; Sec. II A needs a true bound):
 *   0 (default)  max |theta| + beta_{k+1}: the extreme Ritz value plus the
 *                whole residual norm;
 *   1            max |theta| + beta_{k+1} max_i |e_k^T z_i|: the largest
 *                residual of any Ritz pair (z_i the eigenvectors of the
 *                tridiagonal matrix, taken from the interlacing identity
 *                without forming them).
 * Both are times 1.001 and clamped to the Pauli 1-norm. Rule 0 takes the
 * call's lanczos_steps (20 by default); rule 1 runs the same recurrence on to
 * 64 steps (at most 2^N), whose first steps are rule 0's, so rule 0's bound is
 * the same under either rule. Rule 1 then runs about 1.08 times the spectral
 * radius (1.14 at 20 steps) where rule 0 runs about 1.46 (measured against
 * dense spectra). Under rule 1 the KPM moments, the network's features and
 * the window a still come from rule 0's bound (so a network sees the features
 * it was trained on); rule 1's bound becomes E_max of the two recurrences and
 * K is rescaled to K * E_max1 / E_max0: the filter's growth inside the window
 * (exp(2c sqrt(a^2 - E^2) / a), c = K a / E_max) and the basis orders' energy
 * resolution do not depend on E_max, so the filter and evolution lengths
 * shrink in proportion and nothing else changes. Rule 1 is a bound in
 * practice, not in theory: a realization whose moments then exceed mu_0 is
 * reported as DACP_ERR_NUMERIC, and dacp_solve_learned re-runs it under rule 0.
 * Takes effect at the next parameter choice. Errors: DACP_ERR_ARG for another
 * rule.
 */
dacp_status dacp_set_emax_rule(dacp_handle hd, int rule);

/*
 * dacp_test_emax_rule -- test hook (host arithmetic only, no device work): the
 * bound of rule 0 or 1 above, before the safety factor and the clamp, for a
 * k x k Lanczos tridiagonal (1 <= k <= 64): alpha[k] its diagonal, beta2[k] the
 * squared off-diagonals beta_2^2 .. beta_k^2 followed by the squared residual
 * norm beta_{k+1}^2. It is the same code the device kernel runs for rule 1.
 * Errors: DACP_ERR_ARG.
 */
dacp_status dacp_test_emax_rule(int k, const double* alpha, const double* beta2, int rule, double* bound);

/*
 * dacp_set_solver -- how dacp_central_eigs runs the dense float64 algebra:
 * 1 (default) = one batched cuSOLVER syev call per group (up to 256
 * realizations) for S and one for H~, with two strided-batched dgemms
 * (W = H U, H~ = U^T W) between them; smaller bases are
 * zero-padded to the largest (the padding only adds S eigenvalues 0, which
 * the cut-off removes). Used when there are several realizations and every
 * basis is at least 3/4 of the largest. 0 = concurrent lanes (own stream,
 * handles and host thread each) solving the realizations one by one.
 * dacp_solve always uses the batched form, in groups of similar basis size.
 */
dacp_status dacp_set_solver(dacp_handle hd, int mode);

/*
 * dacp_test_poison_barrier -- test hook for the bounded waits: the next
 * persistent launch starts with a grid-barrier arrival count that can never
 * complete, so every CTA's wait gives up after about one second and the call
 * returns DACP_ERR_TIMEOUT with the context still usable. No GPU fault is
 * involved.
 */
dacp_status dacp_test_poison_barrier(dacp_handle hd);

/*
 * dacp_test_fail_alloc -- test hook for allocation failure: after `after`
 * more device allocations by this library (0 = the next one), one allocation
 * fails as if cudaMalloc had run out of memory, and the call that made it
 * returns DACP_ERR_NOMEM after freeing what it allocated (dacp_create frees
 * the whole handle; a handle whose call failed can still be destroyed).
 * Negative `after` switches the hook off; it also switches itself off once
 * it has fired. Process-wide, so it reaches dacp_create. Allocations inside
 * cuSOLVER / cuBLAS and of the parameter network are not counted.
 */
dacp_status dacp_test_fail_alloc(int64_t after);

/*
 * dacp_get_launch_count -- number of this library's own CUDA kernels launched
 * on the handle since dacp_create (kernels inside cuSOLVER / cuBLAS calls are
 * not counted). A graph replay counts each kernel node it runs.
 */
dacp_status dacp_get_launch_count(dacp_handle hd, int64_t* count);

/* ---- learned parameter predictor ------------------------------------------
 * A small float32 MLP (project extension; the paper picks a, K and n by hand,
 * Sec. III). Input: kFeatures = 40 features per realization -- N,
 * log(n_eigs / 2^N), mean/std of the x-fields, of the nonzero zz couplings and
 * of the z-fields, and mu_1..mu_32 of a normalised random vector under
 * G = H / E_max. Output: 3 knobs -- log of the window ratio d / n_eigs, the
 * filter-order constant c (K = c E_max / a) and the basis ratio b(2n+1) / d.
 * Layers: affine + ReLU for the hidden layers, affine output; loss
 * sum (y - t)^2 / (2B) on standardised inputs and targets; Adam.
 * Weights are one flat float32 vector: for each layer W (out x in, row-major)
 * then b. Host arrays passed in are copied; the caller keeps ownership. Every
 * call returns a status (DACP_ERR_ARG for NULL or mis-sized arguments,
 * DACP_ERR_NOMEM, DACP_ERR_CUDA), and a failed call leaves its message in
 * dacp_mlp_last_error. */
typedef struct dacp_mlp_ctx* dacp_mlp;

/* dacp_mlp_create -- layers n_in -> hidden_layers x n_hidden -> n_out.
 * weights: initial flat weights, or NULL for He-uniform weights from seed.
 * stream: cudaStream_t or NULL (private stream). */
dacp_status dacp_mlp_create(dacp_mlp* out, int n_in, int n_hidden, int hidden_layers, int n_out,
                            const float* weights, uint64_t seed, void* stream);
/* dacp_mlp_set_output_range -- clamp every denormalised output y_i to
 * [lo[i], hi[i]] (n_out floats each, host; lo <= hi, else DACP_ERR_ARG).
 * Default: no clamp. A trained network is kept to the range of its labels,
 * so that it never extrapolates to knobs it was not trained on. */
dacp_status dacp_mlp_set_output_range(dacp_mlp m, const float* lo, const float* hi);
/* dacp_mlp_set_normalization -- feature and target standardisation:
 * z = (x - in_mean) / in_std into the network, y = z_out * out_std + out_mean. */
dacp_status dacp_mlp_set_normalization(dacp_mlp m, const float* in_mean, const float* in_std,
                                       const float* out_mean, const float* out_std);
/* dacp_mlp_get_weights / dacp_mlp_set_weights -- copy the flat float32
 * weights to / from caller-owned host memory (set also resets the Adam state).
 * get writes *count (the number of weights, when count is not NULL) and
 * returns DACP_ERR_ARG if cap is smaller. set returns DACP_ERR_ARG unless
 * count equals that number. */
dacp_status dacp_mlp_get_weights(dacp_mlp m, float* w, int64_t cap, int64_t* count);
dacp_status dacp_mlp_set_weights(dacp_mlp m, const float* w, int64_t count);
/* dacp_mlp_forward -- y[batch][n_out] (denormalised) from host x[batch][n_in]. */
dacp_status dacp_mlp_forward(dacp_mlp m, const float* x, int batch, float* y);
/* dacp_mlp_gradients -- gradient of the loss w.r.t. the flat weights for one
 * batch of host (x, t) (targets in raw units), and the loss. Test hook. */
dacp_status dacp_mlp_gradients(dacp_mlp m, const float* x, const float* t, int batch, float* grad,
                               double* loss);
/* dacp_mlp_train -- Adam (lr, beta = 0.9 / 0.999, eps = 1e-8) on shuffled
 * minibatches for `epochs` passes over n_samples host samples; the data is
 * copied to the device once. *final_loss = loss of the last minibatch. */
dacp_status dacp_mlp_train(dacp_mlp m, const float* x, const float* t, int n_samples, int batch,
                           int epochs, float lr, uint64_t seed, double* final_loss);
/* dacp_mlp_get_launch_count -- kernels this network has launched since
 * dacp_mlp_create (forward, backward, loss and Adam kernels). DACP_ERR_ARG for
 * a NULL handle or count. */
dacp_status dacp_mlp_get_launch_count(dacp_mlp m, int64_t* count);
/* dacp_mlp_last_error -- message of the last failed call on m. The string is
 * owned by m and valid until m's next call or its destruction. Returns
 * "NULL handle" for NULL. */
const char* dacp_mlp_last_error(dacp_mlp m);
/* dacp_mlp_destroy -- waits for m's stream, then frees its device buffers and,
 * if m created it, its stream. NULL is ignored. */
void dacp_mlp_destroy(dacp_mlp m);

/*
 * dacp_choose_params_mlp -- parameters from the network: the same Lanczos
 * bound and KPM moments as dacp_choose_params, then the features, one forward
 * pass over all realizations on the device, and the window / order / basis
 * from the predicted knobs (clamped to window ratio [1, 4], c [3, 24],
 * basis ratio [0.6, 3]). The network must have 40 inputs and 3 outputs.
 * dacp_solve_learned runs the path with these parameters and falls back to
 * dacp_choose_params for realizations whose count comes back short.
 */
dacp_status dacp_choose_params_mlp(dacp_handle hd, dacp_mlp m, int n_eigs, int lanczos_steps,
                                   int kpm_moments);

/*
 * dacp_solve_learned -- the whole path with the network's parameters and the
 * heuristic as fallback: dacp_choose_params_mlp (20 Lanczos steps, 256 KPM
 * moments), then dacp_solve; every realization that returns fewer than n_eigs
 * levels (n_found[r] < n_eigs, failures included) is run again with the
 * heuristic of dacp_choose_params (d_ratio 2, basis ratio 1.5, the precision's
 * filter constant, E_max rule 0) on a handle of its own, built from
 * this handle's copies of its couplings, fields, pair couplings and start
 * vectors, on the same stream; its results replace the learned ones.
 *   net         a 40-input, 3-output network (dacp_mlp_create); not modified.
 *   n_eigs, window, eps, eigs, n_found, rank  as in dacp_solve.
 *   n_fallback  may be NULL; the number of realizations re-run.
 * The handle keeps the learned run's state (moments, timings); the re-run's
 * device work is counted in dacp_get_launch_count but not in
 * dacp_get_timings. Errors: as dacp_choose_params_mlp and dacp_solve;
 * a failed re-run returns its status with its message.
 */
dacp_status dacp_solve_learned(dacp_handle hd, dacp_mlp net, int n_eigs, double window, double eps, double* eigs,
                               int* n_found, int* rank, int* n_fallback);

/*
 * dacp_solve_sectors -- the whole path on a dacp_create_parity_sectors handle,
 * with levels per model: each sector is asked for n_sector levels (parameters
 * from `net` with dacp_solve_learned's fallback when net is not NULL, else the
 * Sec. III heuristic under the handle's E_max rule), the two sectors of every
 * model are merged (dacp_merge_sectors), and every model whose merge comes up
 * short of n_eigs -- its sectors split the central levels more unevenly than
 * n_sector allows -- or whose sector failed has both sectors solved again on
 * a handle of their own (E_max rule 0, the heuristic), each asked for all
 * n_eigs levels, which the union then always covers.
 *   n_eigs     levels wanted per model; n_sector in [1, n_eigs] per sector
 *              (the central levels split about evenly: a little above
 *              n_eigs / 2 is enough almost always).
 *   eigs       [R/2][n_eigs] float64 host buffer, n_found [R/2] host ints
 *              (as dacp_merge_sectors writes them).
 *   n_redone   models solved again (may be NULL).
 * Errors: DACP_ERR_ARG for a handle not made by dacp_create_parity_sectors or
 * bad sizes; the errors of dacp_solve / dacp_solve_learned.
 */
dacp_status dacp_solve_sectors(dacp_handle hd, dacp_mlp net, int n_eigs, int n_sector, double* eigs, int* n_found,
                               int* n_redone);

/* dacp_get_features -- the 40 network features of every realization
 * (float32, [n_real][40]) from the last parameter choice. */
dacp_status dacp_get_features(dacp_handle hd, float* feats, int64_t cap);

/*
 * dacp_moments_noalloc -- Chebyshev moments of one realization without any
 * device allocation. The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- engines whose device memory all comes
 * from their own pool or arena (a cudaMalloc behind their back would break
 * their accounting or fail under their memory cap), and loops that must not
 * enter an allocator (an allocation can synchronize the device and stall
 * them).
 *
 *   n_spins      N, 1 <= N <= 16; larger N returns DACP_ERR_ARG (the scratch
 *                array below holds 3 x 2^16 float64 states).
 *   J, h, gamma  host arrays as in dacp_create for one realization (J is
 *                N x N row-major, only i<j read).
 *   emax         bound on |E|; G = H / emax.
 *   psi_dev      device pointer, 2^N float64: the start vector (used as given,
 *                not normalised).
 *   n_orders     evolution orders k = 0 .. n_orders-1.
 *   mu_dev       device pointer, 2 * n_orders float64: on return
 *                mu_j = <psi| T_j(G) |psi>, j = 0 .. 2 n_orders - 1, from the
 *                same fused stencil kernel as dacp_basis_moments.
 *   stream       cudaStream_t or NULL. The call copies J, h, gamma and its
 *                run lengths from host memory into the scratch array on this
 *                stream, and waits for the stream before it returns.
 *
 * Scratch: one file-scope device array of about 1.6 MB (vectors, diagonal,
 * couplings, partial sums, counters), held by every GPU that loads the
 * library until the process exits. The first call on a device does the
 * set-up: it looks up the array's address (cudaGetSymbolAddress) and raises
 * the stencil kernel's shared-memory limit; make that first call before any
 * stream capture. Every call overwrites the array and clears its counters,
 * and two calls that overlap on the GPU (different streams or threads) race
 * on it and corrupt each other's results: serialise them.
 * Returns DACP_OK, DACP_ERR_ARG, DACP_ERR_CUDA or DACP_ERR_TIMEOUT.
 */
dacp_status dacp_moments_noalloc(int n_spins, const double* J, const double* h, const double* gamma,
                                 double emax, const double* psi_dev, int n_orders, double* mu_dev,
                                 void* stream);

/* dacp_last_error -- message of the last failure on this handle (owned by
 * the handle, valid until the next call on it). */
const char* dacp_last_error(dacp_handle hd);

/* dacp_status_string -- static name of a status code. */
const char* dacp_status_string(int status);

/* dacp_destroy -- free every device buffer of the handle. NULL is allowed. */
void dacp_destroy(dacp_handle hd);

#ifdef __cplusplus
}
#endif

#endif /* DACP_H */
