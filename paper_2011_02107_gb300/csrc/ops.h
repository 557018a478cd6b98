// Host-side launchers of the DACP kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace dacp {

// stencil.cu
cudaError_t prepare_step(int prec, int b, int smem);
cudaError_t launch_persistent(int prec, int b, int seq, const StepArgs& a, int n_items, int orders, int smem,
                              cudaStream_t st, int* grid_out);
cudaError_t launch_step(int prec, int b, int mode, const StepArgs& a, int item_base, int n_items, int smem,
                        cudaStream_t st);
// float32 only: recurrence passes with the tile's x, y and diagonal staged by bulk copies
int staged_smem_bytes(int mode, int b, int tile_smem);
bool staged_fits(int b, int tile_smem);
cudaError_t prepare_step_staged(int b, int tile_smem);
cudaError_t launch_step_staged(int b, int mode, const StepArgs& a, int item_base, int n_items, int tile_smem,
                               cudaStream_t st);
cudaError_t launch_diag(int prec, const RealInfo* real, int r, int N, const double* J, const double* h,
                        void* diag, cudaStream_t st);
cudaError_t launch_diag_all(int prec, const RealInfo* real, int R, int max_N, const double* J, const double* h,
                            void* diag, cudaStream_t st);
cudaError_t launch_scatter_convert(int prec, const double* src, const int64_t* src_off, const RealInfo* real, int R,
                                   int max_N, int b, void* dst, cudaStream_t st);
cudaError_t launch_convert(int prec, const double* src, void* dst, int64_t n, cudaStream_t st);
cudaError_t launch_to_double(int prec, const void* src, double* dst, int64_t n, int b, cudaStream_t st);
cudaError_t launch_gather_basis(int prec, int b, const void* src, int64_t D, double* V, int64_t ldv, int col0,
                                cudaStream_t st);
cudaError_t launch_normalize(int prec, int b, const Item* items, const RealInfo* real, int n_items,
                             const void* A, const void* Bv, int by_parity, double* part, unsigned* real_done,
                             double* norms, void* dst, void* dst2, cudaStream_t st);
cudaError_t launch_extract_col(int prec, int b, const void* src, void* dst, int64_t states, cudaStream_t st);

// subspace.cu
cudaError_t launch_orders(int L, double a_r, int* orders, cudaStream_t st);
cudaError_t launch_moments(const double* P, int rows, int b, double emax, double* mus, double* nus, int* bad,
                           cudaStream_t st);
cudaError_t launch_assemble(int L, int b, const int* orders, const double* mus, const double* nus, double* S,
                            double* H, cudaStream_t st, int ld = 0);
cudaError_t launch_cutoff(const double* lam, int M, double eps, int absolute, double* V, int* m_out,
                          cudaStream_t st);
cudaError_t launch_select(const double* lam, int m, int n_eigs, double w, double* out, int* n_found,
                          cudaStream_t st);
cudaError_t launch_omega(const double* mus, int rows_out, int b, double emax, double* om, cudaStream_t st);
cudaError_t launch_select_range(const double* lam, int m, int n_eigs, double w, int* out, cudaStream_t st);
cudaError_t launch_residual(const double* Bsel, const double* W2, int M, int count, const double* lam, double* resid,
                            cudaStream_t st);
cudaError_t launch_pad_columns(double* V, int M, int64_t strideV, const int* m, int m_max, int count, cudaStream_t st);
cudaError_t launch_pad_diagonal(double* Ht, int m_max, int64_t strideH, const int* m, const double* big, int count,
                                cudaStream_t st);
cudaError_t launch_ritz_residual(const double* HY, const double* Y, const double* th, int64_t D, int m, double* res,
                                 cudaStream_t st);
cudaError_t launch_compact_converged(const double* th, const double* res, int m, double tol, double* out, int* count,
                                     cudaStream_t st);

// params.cu
cudaError_t launch_lanczos_orth(int prec, const Item* items, const RealInfo* real, int n_items, const void* v,
                                void* w, const double* lmom, int rows, int j, double* part, unsigned* real_done,
                                double* beta2, int steps, cudaStream_t st);
cudaError_t launch_lanczos_scale(int prec, const Item* items, const RealInfo* real, int n_items, void* w,
                                 const double* beta2, int j, int steps, double* coef, int R, cudaStream_t st);
cudaError_t launch_lanczos_bound(int R, const double* lmom, int rows, const double* beta2, int steps, int stride,
                                 const double* pnorm, double safety, double* emax, int rule, cudaStream_t st);
cudaError_t launch_kpm_window(int R, const RealInfo* real, const double* P, int M, const double* emax,
                              double d_target, double c_order, double basis_ratio, int b, const float* knobs,
                              int n_eigs, double* a_out, int* K_out, int* n_out, cudaStream_t st);
cudaError_t launch_features(int R, const RealInfo* real, const double* J, const double* h, const double* g,
                            const double* P, int M, int n_eigs, float* out, cudaStream_t st);

// mlp.cu
}  // namespace dacp

struct dacp_mlp_ctx;

namespace dacp {
cudaError_t mlp_forward_device(struct dacp_mlp_ctx* m, const float* feats, int B, float* out, cudaStream_t st,
                               int64_t* launches);
int mlp_n_in(struct dacp_mlp_ctx* m);
int mlp_n_out(struct dacp_mlp_ctx* m);
}  // namespace dacp
