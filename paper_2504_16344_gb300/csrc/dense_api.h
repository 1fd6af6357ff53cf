// dense_api.h -- host launchers of dense.cu (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "dense.cuh"

namespace tw {

// P = G G^T (lower 64x64 tiles) into K (FP64); G: [n][kdim] dd, row stride ldg.
// Tensor cores with exact bf16 slices of G (gemm_syrk.cu): tl = the tile list
// of syrk_tile_list(n_pad) in device memory, eg syrk_exp_rows(n_pad) ints, ws
// a multiple of syrk_ws_bytes_per_atom(n_pad) bytes (at least 4 of them)
void syrk_tile_list(int n_pad, std::vector<int2> &tl);
size_t syrk_ws_bytes_per_atom(int n_pad);
int syrk_exp_rows(int n_pad);
cudaError_t launch_syrk_update_d(const double *A, long lda, int kdim, double *C, long ldc, int m,
                                 uint8_t *ws, size_t ws_bytes, int *eg, int *err, cudaStream_t s);
int cholesky_tc_width();   // block columns per tensor-core trailing update
cudaError_t launch_form_P_tc(const dd *G, long ldg, int n, int kdim, double *K, long ldk, int n_pad,
                             uint8_t *ws, size_t ws_bytes, int *eg, const int2 *tl, int ntl, int *err,
                             cudaStream_t s);
// K = sigma2 I + block-diagonal prefix sums of P (in place, FP64), identity padding
cudaError_t launch_K_from_P(double *K, long ldk, int Nd, int Nt, int n, int n_pad, double sigma2,
                            cudaStream_t s);
// blocked Cholesky in place (lower), inverses of the diagonal blocks to inv
cudaError_t launch_cholesky_f(float *K, long ldk, int NB, float *inv, int *err, cudaStream_t s);
// FP64: the trailing updates on the tensor cores with slice workspaces ws
// (>= syrk_ws_bytes_per_atom(64 NB) * 2 * cholesky_tc_width() bytes) and eg
// (>= syrk_exp_rows(64 NB) ints); ws = nullptr keeps them on the FP64 pipe
cudaError_t launch_cholesky_d(double *K, long ldk, int NB, double *inv, int *err, uint8_t *ws,
                              size_t ws_bytes, int *eg, cudaStream_t s);
cudaError_t launch_pack_d(const double *K, long ldk, double *P, int NB, cudaStream_t s);
cudaError_t launch_pack_d2dd(const double *K, long ldk, dd *P, int NB, cudaStream_t s);
cudaError_t launch_double_to_dd(const double *a, dd *b, size_t n, cudaStream_t s);
cudaError_t launch_pack_f(const float *K, long ldk, float *P, int NB, cudaStream_t s);
cudaError_t launch_lower_to_float(const double *K, float *K32, long ld, int NB, cudaStream_t s);

// FP64-class solves of one right-hand side with the block-scaled factor,
// stored as float pairs, in double-float arithmetic (trsv64.cu)
struct Trsv64Args {
  const dd *Lf, *Lb;                // packed Linv_I L_IJ and L_IJ Linv_J (J < I)
  const double *Linv;               // [NB][64][64] diagonal-block inverses (FP64)
  const dd *bands;                  // [2][DCH][NB][64][64] chain blocks as split planes:
                                    //   FWD Lf_{I,I-j}^T, BWD Lb_{I+j,I}
  int NB;                           // block rows of the factor (bands' stride)
  const void *rhs;                  // kind 0 double, 1 float pairs; must not alias outx
  int rhs_kind;
  double *out;                      // [>= NBw*64] the solution (rows >= nrows set to 0)
  dd *outx;                         // [>= NBw*64] the same as float pairs (read by the workers)
  int nrows, NBw;
  const int2 *tasks;                // (row, chunk) in row order; tasks of rows < NBw form a prefix
  int ntasks;
  dd *part;                         // [NB][maxk][64] partial sums
  int maxk;
  int *cnt;                         // [NB] tasks done per row, zeroed by the launcher
  dd *wbuf;                         // [n_pad] w_u hand-off, filled with all-ones by the launcher
  int *prog, *err, *abort_flag;     // prog: 2 ints, zeroed by the launcher
};
int trsv64_max_tasks_per_row(int NB);
void trsv64_task_table(int NB, std::vector<int> &tab, std::vector<int> &prefix);
int trsv64_chain_deps();            // DCH: dependencies the chain CTA applies
cudaError_t launch_trsv64_setup(const double *Lp, const double *Linv, dd *Lf, dd *Lb, dd *bands,
                                int NB, cudaStream_t s);
cudaError_t launch_trsv64(const Trsv64Args &a, bool fwd, cudaStream_t s);
// triangular solves (fwd: L z = b; bwd: L^T x = z), rhs kind 0 double / 1 dd / 2 float
// prog: two ints (ticket, rows finished), zeroed by the launcher
// Lchain: M_I = Linv_I L_{I,I-1} (fwd) or C_I = L_{I+1,I} Linv_I (bwd), [NB][64][64]
cudaError_t launch_trsv_f(const float *Lp, const float *Linv, const float *Lchain,
                          const void *rhs, int rhs_kind, float *out, int nrows, int NBw, int *prog,
                          bool fwd, int *err, int *abort_flag, cudaStream_t s);
// batched solves (B right-hand sides, column b at rhs + b*rhs_bstride /
// out + b*out_bstride, window win[b] time steps in device memory); prog:
// trsm_prog_ints(B) ints, zeroed by the launcher
int trsm_prog_ints(int B);
cudaError_t launch_trsm_d(const double *Lp, const double *Linv, const double *Lchain,
                          const void *rhs, int rhs_kind, long rhs_bstride, double *out,
                          long out_bstride, const int *win, int Nd, int Nt, int B, int NB,
                          int *prog, bool fwd, int *err, int *abort_flag, cudaStream_t s);
// the same sweeps with the single-vector solve's pre-multiplied blocks: Lx =
// Lf (Linv_I L_IJ, forward) or Lb (L_IJ Linv_J, backward), packed like L
cudaError_t launch_trsm_dd_scaled(const dd *Lx, const dd *Linv, const void *rhs, int rhs_kind,
                                  long rhs_bstride, dd *out, long out_bstride, const int *win, int Nd,
                                  int Nt, int B, int NB, int *prog, bool fwd, int *err, int *abort_flag,
                                  cudaStream_t s);
cudaError_t launch_chain_blocks_d(const double *Lp, const double *Linv, double *Mf, double *Cb,
                                  int NB, cudaStream_t s);
cudaError_t launch_chain_blocks_f(const float *Lp, const float *Linv, float *Mf, float *Cb, int NB,
                                  cudaStream_t s);
// r = d - K x (packed lower K, df64); d == nullptr gives r = K x
cudaError_t launch_residual(const dd *Kp, const dd *x, const double *d, dd *r, int nrows, int NBw,
                            cudaStream_t s);
cudaError_t launch_dd_to_double(const dd *a, double *b, int n, cudaStream_t s);
cudaError_t launch_double_to_dd_vec(const double *a, dd *b, int n, cudaStream_t s);
cudaError_t launch_sample_rhs(const double *d, const double *a, const double *z, double sigma,
                              double *r, int n, cudaStream_t s);
cudaError_t launch_add_dd(double *sv, const dd *x, long n, cudaStream_t s);
cudaError_t launch_axpy_dd_f(dd *x, const float *delta, int n, cudaStream_t s);
cudaError_t launch_f_to_dd(const float *a, dd *b, int n, cudaStream_t s);
cudaError_t launch_sumsq(const void *v, int kind, int n, double *out, cudaStream_t s);

}  // namespace tw
