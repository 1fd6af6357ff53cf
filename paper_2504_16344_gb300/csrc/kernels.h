// kernels.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fft_engine.cuh"

namespace tw {

// process-wide count of kernels this library has enqueued
void count_launches(int k);
long long launches_total();

// ---- batches of right-hand sides ----------------------------------------
// Entry b of a batch is at base + b * stride (elements of the array's type);
// its window (time steps kept, rows read) is win[b] when win != nullptr,
// capped by the call's scalar window.  win lives in device memory.
struct BatchArg {
  int count = 1;
  long in_stride = 0, out_stride = 0, work_stride = 0;
  const int *win = nullptr;
  __device__ __forceinline__ int window(int b, int cap) const {
    return win ? min(max(win[b], 0), cap) : cap;
  }
};

// ---- operator storage formats
enum OpFmt { FMT_DD = 0, FMT_C64 = 1, FMT_BF16X2 = 2 };

// ---- time-axis real FFT (length 2M, second half zero) -------------------
// in  [M rows][N series] real, row stride in_ld; rows >= n_in treated as 0
// out [M+1 rows][N] complex, row stride out_ld
// in_kind: 0 = double, 1 = dd (float2), 2 = float
cudaError_t launch_rfft_time_dd(const void *in, int in_kind, long in_ld, int n_in,
                                cdd *out, long out_ld, int N, const FftPlan &pl,
                                const cdd *twM, const cdd *twL, cudaStream_t s,
                                const BatchArg &ba = BatchArg{});
cudaError_t launch_rfft_time_f(const void *in, int in_kind, long in_ld, int n_in,
                               cf *out, long out_ld, int N, const FftPlan &pl,
                               const cf *twM, const cf *twL, cudaStream_t s,
                               const BatchArg &ba = BatchArg{});
// inverse: in [M+1][N] complex -> out [M][N] real (1/(2M) applied),
// rows t >= n_keep written as 0.  out_kind: 0 = double, 1 = dd, 2 = float
cudaError_t launch_irfft_time_dd(const cdd *in, long in_ld, void *out, int out_kind, long out_ld,
                                 int N, int n_keep, const FftPlan &pl, const cdd *twM,
                                 const cdd *twL, cudaStream_t s, const BatchArg &ba = BatchArg{});
cudaError_t launch_irfft_time_f(const cf *in, long in_ld, void *out, int out_kind, long out_ld,
                                int N, int n_keep, const FftPlan &pl, const cf *twM,
                                const cf *twL, cudaStream_t s, const BatchArg &ba = BatchArg{});
// inverse as above (out: m, rows t >= n_keep zero), then the forward transform
// of that m (zero-padded, as launch_rfft_time_*) into spec [M+1][N]; spec may be
// in.  Batches: right-hand side b reads in + b * ba.in_stride, writes m at
// out + b * ba.out_stride and its spectrum at spec + b * ba.work_stride, with
// window ba.window(b, n_keep)
cudaError_t launch_irfft_rfft_time_dd(const cdd *in, long in_ld, void *out, int out_kind, long out_ld,
                                      cdd *spec, long spec_ld, int N, int n_keep, const FftPlan &pl,
                                      const cdd *twM, const cdd *twL, cudaStream_t s,
                                      const BatchArg &ba = BatchArg{});
cudaError_t launch_irfft_rfft_time_f(const cf *in, long in_ld, void *out, int out_kind, long out_ld,
                                     cf *spec, long spec_ld, int N, int n_keep, const FftPlan &pl,
                                     const cf *twM, const cf *twL, cudaStream_t s,
                                     const BatchArg &ba = BatchArg{});

// ---- Matern filter on the periodic grid: y_t = C^power x_t, t < nt -------
// x, y: [nt][Nx][Ny] real (kind 0 double, 1 dd, 2 float); work: [ceil(nt/2)][Nx][Ny] complex
// lam: [Nx][Ny] eigenvalues^power / (Nx Ny)
// batched: entry b reads x + b*ba.in_stride, writes y + b*ba.out_stride, uses
// work + b*ba.work_stride; accum != 0 adds the result to y instead of storing it
cudaError_t launch_prior_dd(const void *x, int in_kind, void *y, int out_kind, int nt, int Nx,
                            int Ny, cdd *work, const dd *lam, const FftPlan &plx,
                            const FftPlan &ply, const cdd *twx, const cdd *twy, cudaStream_t s,
                            const BatchArg &ba = BatchArg{}, int accum = 0);
// native FP64 variant (set-up); output field t goes to (t/per)*stride + off + t%per
cudaError_t launch_prior_d(const void *x, int in_kind, void *y, int out_kind, int nt, int Nx,
                           int Ny, cd *work, const double *lam, const FftPlan &plx,
                           const FftPlan &ply, const cd *twx, const cd *twy, int map_per,
                           int map_stride, int map_off, cudaStream_t s);
// x[f] <- C x[f] for complex fields f < nf (cdd storage, FP64 arithmetic, set-up);
// lam: eigenvalues / (Nx Ny) in FP64; work: nf_chunk fields of cd
cudaError_t launch_prior_cfields_d(cdd *x, long nf, int Nx, int Ny, cd *work, long nf_chunk,
                                   const double *lam, const FftPlan &plx, const FftPlan &ply,
                                   const cd *twx, const cd *twy, cudaStream_t s);
cudaError_t launch_prior_f(const void *x, int in_kind, void *y, int out_kind, int nt, int Nx,
                           int Ny, cf *work, const float *lam, const FftPlan &plx,
                           const FftPlan &ply, const cf *twx, const cf *twy, cudaStream_t s,
                           const BatchArg &ba = BatchArg{}, int accum = 0);

// ---- frequency-batched complex GEMV ------------------------------------
// forward: yh[w][s] = sum_k A[w][s][k] xh[w][k]   (A: [Nf][Nr][Nm] in `fmt`)
// partial sums per k-chunk go to `part` ([Nf][nchunk][Nr]) then are reduced.
int gemv_fwd_nchunk(int Nm);
cudaError_t launch_gemv_fwd_dd(const void *A, int fmt, const cdd *xh, cdd *part, cdd *yh,
                               int Nf, int Nr, int Nm, cudaStream_t s);
cudaError_t launch_gemv_fwd_f(const void *A, int fmt, const cf *xh, cf *part, cf *yh, int Nf,
                              int Nr, int Nm, cudaStream_t s);
// adjoint: xh[w][k] = sum_s conj(A[w][s][k]) yh[w][s]
cudaError_t launch_gemv_adj_dd(const void *A, int fmt, const cdd *yh, cdd *xh, int Nf, int Nr,
                               int Nm, cudaStream_t s);
// adjoint for one right-hand side with an FP32 operator (fmt C64 / BF16X2)
// and float-pair data: exact products, double-float running sums, x^ in FP32
cudaError_t launch_gemv_adj_cx(const void *A, int fmt, const cdd *yh, cf *xh, int Nf, int Nr, int Nm,
                               cudaStream_t s);

// ---- batched per-frequency products (gemm.cu) ----------------------------
// adjoint: X[b][w][k] = sum_s conj(A[w][s][k]) Y[b][w][s]
// forward: Yo[b][w][r] = sum_k A[w][r][k] X[b][w][k]; part: B*Nf*nchunk*Nr entries
int gemm_fwd_nchunk(int Nm);
// rw: right-hand sides per warp (1, 2 or 4; 0 picks after B).  Each column's
// sum runs over the rows in the same order whatever rw is.
cudaError_t launch_gemm_adj_dd(const void *A, const cdd *Y, long y_bstride, cdd *X, long x_bstride,
                               int Nf, int Nr, int Nm, int B, cudaStream_t s, int rw = 0);
// lpb: lanes per right-hand side in the forward product (1 or 2, fixed per
// context so that a right-hand side's sum order does not depend on its batch)
cudaError_t launch_gemm_fwd_dd(const void *A, const cdd *X, long x_bstride, cdd *part, cdd *Yo,
                               long y_bstride, int Nf, int Nr, int Nm, int B, cudaStream_t s, int lpb = 1);
cudaError_t launch_gemm_fwd_f(const void *A, int fmt, const cf *X, long x_bstride, cf *part,
                              cf *Yo, long y_bstride, int Nf, int Nr, int Nm, int B,
                              cudaStream_t s, int lpb = 1);

// ---- reduced-precision adjoint product on the tensor cores (gemm_sl.cu) ---
// X[b][w][k] = sum_s conj(A[w][s][k]) Y[b][w][s] with the FP32 operator
// (fmt C64 / BF16X2) and float-pair data Y, both cut into exact fixed-point
// bf16 slices; ea: the operator's row exponents (launch_row_exp).  P: right-
// hand sides per tile (multiple of 8, <= 80; 0 picks one).  ws / eb: the
// data-side slices and exponents, at least sl_ws_bytes / sl_eb_bytes for
// ceil(B / P) P columns.  err: device error record (bounded waits).
int sl_natoms(int Nr);
size_t sl_ws_bytes(int Nf, int Nr, int bcols);
size_t sl_eb_bytes(int Nf, int bcols);
int sl_pick_tile(int B);
cudaError_t launch_row_exp(const void *A, int fmt, int8_t *ea, int Nf, int Nr, int Nm, cudaStream_t s);
cudaError_t launch_gemm_adj_sl(const void *A, int fmt, const int8_t *ea, const cdd *Y, long y_bstride,
                               cf *X, long x_bstride, int Nf, int Nr, int Nm, int B, int P,
                               void *ws, size_t ws_bytes, int *eb, size_t eb_bytes, int *err,
                               cudaStream_t s);

// ---- operator storage conversion: dst[w][row0+r][k] from src (cdd) -----
cudaError_t launch_convert_op(const cdd *src, long src_ld_w, void *dst, int fmt, long dst_ld_w,
                              long n_per_w, int Nf, cudaStream_t s);

}  // namespace tw
