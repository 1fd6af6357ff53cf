// qoi.cu -- Phase 3 precomputations for the QoI and the Phase 4 map q = Q d.
//
// Phase 3 of the framework (Sec. "Real-time Bayesian inference and
// prediction framework") forms, from Nq Nt actions on QoI unit vectors,
//   the data-to-QoI map        Q = F_q Gamma_post F^* Gamma_n^{-1}
//   the QoI posterior covariance  Gamma_post(q) = F_q Gamma_post F_q^*
// so that Phase 4 predicts q = Q d without reconstructing m.  With the
// data-space Hessian K = Gamma_n + F Gamma_pr F^* these are
//   Q = F_q Gamma_pr F^* K^{-1}          (push-through identity)
//   Gamma_post(q) = C - W^T K^{-1} W,    C = F_q Gamma_pr F_q^*,  W = F Gamma_pr F_q^*.
// For a batch of unit vectors e_j (QoI entry j = t Nq + i) the build runs
//   u_j = Gamma_pr F_q^T e_j     (batched adjoint with F_q^, prior filter)
//   c_j = F_q u_j,  w_j = F u_j  (one time FFT of u_j feeds both products)
//   y_j = K^{-1} w_j             (batched triangular solves)
// and keeps Q (row j = y_j), W (row j = w_j), C (row j = c_j) and the
// variances C_jj - w_j . y_j (batches of up to 96).  FP64 path throughout (double-float applies,
// FP64 factor); the full covariance is one FP64 GEMM on request.
#include <algorithm>
#include <vector>

#include "ctx.h"
#include "dense_api.h"

using namespace tw;

namespace {

__global__ void k_unit_qoi(double *__restrict__ e, int nq, int j0, int B) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)B * nq) return;
  const int b = (int)(i / nq), j = (int)(i % nq);
  e[i] = (j == j0 + b) ? 1.0 : 0.0;
}

__global__ void k_fill_int(int *a, int v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// var[j0+b] = C[b][j0+b] - sum_i y[b][i] w[b][i]   (one CTA per b)
__global__ void k_qoi_var(const double *__restrict__ cq, const double *__restrict__ y, long y_ld,
                          const double *__restrict__ w, int n, int nq, int j0,
                          double *__restrict__ var) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(y[(size_t)b * y_ld + i], w[(size_t)b * n + i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    var[j0 + b] = cq[(size_t)b * nq + j0 + b] - t;
  }
}

// q[r][j] = sum_i Q[j][i] d[r][i]: one warp per row j, up to 4 right-hand
// sides per pass; eight independent loads per lane in flight (the row is
// streamed once per pass, FP64 FMA)
__global__ void __launch_bounds__(256)
k_qoi_apply(const double *__restrict__ Qm, const double *__restrict__ d, double *__restrict__ q,
            int nq, int n, int nrhs) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nq) return;
  const double *row = Qm + (size_t)warp * n;
  for (int r0 = 0; r0 < nrhs; r0 += 4) {
    const int nr = min(4, nrhs - r0);
    double acc[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r) { acc[r][0] = 0.0; acc[r][1] = 0.0; }
    int i = lane;
    for (; i + 7 * 32 < n; i += 8 * 32) {
      double a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = __ldcs(row + i + 32 * k);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (r >= nr) break;
        const double *dr = d + (size_t)(r0 + r) * n + i;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[r][k & 1] = fma(a[k], __ldg(dr + 32 * k), acc[r][k & 1]);
      }
    }
    for (; i < n; i += 32) {
      const double a = __ldcs(row + i);
      for (int r = 0; r < nr; ++r) acc[r][0] = fma(a, __ldg(d + (size_t)(r0 + r) * n + i), acc[r][0]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      double v = acc[r][0] + acc[r][1];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && r < nr) q[(size_t)(r0 + r) * nq + warp] = v;
    }
  }
}

// G = C - W Q^T  ([nq][nq]; W, Q: [nq][n] rows).  64x64 tiles, 4x4 per thread, FP64.
__global__ void __launch_bounds__(256)
k_qoi_cov(const double *__restrict__ C, const double *__restrict__ W, const double *__restrict__ Qm,
          double *__restrict__ G, int nq, int n) {
  __shared__ double sa[32][65], sb[32][65];
  const int ti = blockIdx.y * 64, tj = blockIdx.x * 64;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      const int r = e >> 5, k = e & 31;
      const int gi = ti + r, gj = tj + r, gk = k0 + k;
      sa[k][r] = (gi < nq && gk < n) ? W[(size_t)gi * n + gk] : 0.0;
      sb[k][r] = (gj < nq && gk < n) ? Qm[(size_t)gj * n + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = sa[k][tr * 4 + u]; b[u] = sb[k][tc * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gi = ti + tr * 4 + u, gj = tj + tc * 4 + v;
      if (gi < nq && gj < nq) G[(size_t)gi * nq + gj] = C[(size_t)gi * nq + gj] - acc[u][v];
    }
}

}  // namespace

extern "C" {

tw_status tw_qoi_build(tw_ctx *c, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (!c->have64 || !c->op[TW_MAP_F][TW_PREC_FP64] || !c->op[TW_MAP_FQ][TW_PREC_FP64])
    return twh::fail(c, TW_ERR_STATE, "tw_qoi_build needs the FP64 operators and factor");
  if (c->lane.bmax <= 0) return twh::fail(c, TW_ERR_STATE, "tw_reserve_batch must come first");
  for (char l : c->loaded[TW_MAP_FQ])
    if (!l) return twh::fail(c, TW_ERR_STATE, "block column of F_q not fully loaded");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int Nd = c->Nd, Nq = c->Nq, Nt = c->Nt, Nm = c->Nm, Nf = c->Nf;
  const int nq = Nq * Nt, n = Nd * Nt;
  const long np = c->n_pad;
  const int Bq = std::min(c->lane.bmax, 96);
  auto need = [&](void *&p, size_t bytes) { if (!p) p = twh::dalloc(c, bytes); return p != nullptr; };
  bool ok = need((void *&)c->Qmap, (size_t)nq * n * sizeof(double)) &&
            need((void *&)c->Wmap, (size_t)nq * n * sizeof(double)) &&
            need((void *&)c->Cqq, (size_t)nq * nq * sizeof(double)) &&
            need((void *&)c->qvar, (size_t)nq * sizeof(double));
  double *eq = (double *)twh::dalloc(c, (size_t)Bq * nq * sizeof(double));
  double *cq = (double *)twh::dalloc(c, (size_t)Bq * nq * sizeof(double));
  double *u = (double *)twh::dalloc(c, (size_t)Bq * Nt * Nm * sizeof(double));
  auto cleanup = [&]() { twh::dfree(c, eq); twh::dfree(c, cq); twh::dfree(c, u); };
  if (!ok || !eq || !cq || !u) { cleanup(); return twh::fail(c, TW_ERR_OOM, "QoI map buffers"); }
  const void *AF = c->op[TW_MAP_F][TW_PREC_FP64], *AQ = c->op[TW_MAP_FQ][TW_PREC_FP64];
  int *prog_f = c->lane.trsm_prog, *prog_b = c->lane.trsm_prog + trsm_prog_ints(c->lane.bmax);
  k_fill_int<<<(Bq + 255) / 256, 256, 0, s>>>(c->lane.win_dev, Nt, Bq);
  count_launches(1);
  for (int j0 = 0; j0 < nq; j0 += Bq) {
    const int B = std::min(Bq, nq - j0);
    const BatchArg ba_e{B, (long)nq, (long)Nf * Nq, 0, nullptr};
    const BatchArg ba_u{B, (long)Nf * Nm, (long)Nt * Nm, 0, nullptr};
    const BatchArg ba_p{B, (long)Nt * Nm, (long)Nt * Nm, (long)((Nt + 1) / 2) * Nm, nullptr};
    const BatchArg ba_r{B, (long)Nt * Nm, (long)Nf * Nm, 0, nullptr};
    const BatchArg ba_q{B, (long)Nf * Nq, (long)nq, 0, nullptr};
    const BatchArg ba_d{B, (long)Nf * Nd, (long)n, 0, nullptr};
    const long ne = (long)B * nq;
    k_unit_qoi<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(eq, nq, j0, B);
    count_launches(1);
    // u = Gamma_pr F_q^T e
    TW_CUDA(c, launch_rfft_time_dd(eq, 0, Nq, Nt, (cdd *)c->lane.byh, Nq, Nq, c->plT, c->twT, c->twL, s, ba_e));
    TW_CUDA(c, launch_gemm_adj_dd(AQ, (const cdd *)c->lane.byh, (long)Nf * Nq, (cdd *)c->lane.bxh, (long)Nf * Nm,
                                  Nf, Nq, Nm, B, s));
    TW_CUDA(c, launch_irfft_time_dd((const cdd *)c->lane.bxh, Nm, u, 0, Nm, Nm, Nt, c->plT, c->twT, c->twL, s, ba_u));
    TW_CUDA(c, launch_prior_dd(u, 0, u, 0, Nt, c->Nx, c->Ny, (cdd *)c->lane.bxh, c->lam1, c->plX, c->plY,
                               c->twX, c->twY, s, ba_p, 0));
    // spectra of u, then c = F_q u and w = F u
    TW_CUDA(c, launch_rfft_time_dd(u, 0, Nm, Nt, (cdd *)c->lane.bxh, Nm, Nm, c->plT, c->twT, c->twL, s, ba_r));
    TW_CUDA(c, launch_gemm_fwd_dd(AQ, (const cdd *)c->lane.bxh, (long)Nf * Nm, (cdd *)c->lane.bpart, (cdd *)c->lane.byh,
                                  (long)Nf * Nq, Nf, Nq, Nm, B, s));
    TW_CUDA(c, launch_irfft_time_dd((const cdd *)c->lane.byh, Nq, cq, 0, Nq, Nq, Nt, c->plT, c->twT, c->twL, s, ba_q));
    TW_CUDA(c, launch_gemm_fwd_dd(AF, (const cdd *)c->lane.bxh, (long)Nf * Nm, (cdd *)c->lane.bpart, (cdd *)c->lane.byh,
                                  (long)Nf * Nd, Nf, Nd, Nm, B, s));
    TW_CUDA(c, launch_irfft_time_dd((const cdd *)c->lane.byh, Nd, c->lane.brd, 0, Nd, Nd, Nt, c->plT, c->twT, c->twL, s, ba_d));
    // y = K^{-1} w
    TW_CUDA(c, launch_trsm_d(c->Lp64, c->inv64, c->chF64, c->lane.brd, 0, (long)n, c->lane.bz, np, c->lane.win_dev, Nd,
                             Nt, B, c->NB, prog_f, true, c->d_err, c->abort_flag, s));
    TW_CUDA(c, launch_trsm_d(c->Lp64, c->inv64, c->chB64, c->lane.bz, 0, np, c->lane.by, np, c->lane.win_dev, Nd, Nt, B,
                             c->NB, prog_b, false, c->d_err, c->abort_flag, s));
    // rows of Q, W, C and the variances
    TW_CUDA(c, cudaMemcpy2DAsync(c->Qmap + (size_t)j0 * n, (size_t)n * sizeof(double), c->lane.by,
                                 (size_t)np * sizeof(double), (size_t)n * sizeof(double), B,
                                 cudaMemcpyDeviceToDevice, s));
    TW_CUDA(c, cudaMemcpyAsync(c->Wmap + (size_t)j0 * n, c->lane.brd, (size_t)B * n * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
    TW_CUDA(c, cudaMemcpyAsync(c->Cqq + (size_t)j0 * nq, cq, (size_t)B * nq * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
    k_qoi_var<<<B, 256, 0, s>>>(cq, c->lane.by, np, c->lane.brd, n, nq, j0, c->qvar);
    count_launches(1);
    TW_CUDA(c, cudaGetLastError());
  }
  TW_CUDA(c, cudaStreamSynchronize(s));
  cleanup();
  tw_status st = tw_check(c, stream);
  if (st == TW_OK) c->have_qoi = true;
  return st;
}

tw_status tw_qoi_apply(tw_ctx *c, int nrhs, const double *d, double *q, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (!c->have_qoi) return twh::fail(c, TW_ERR_STATE, "tw_qoi_build must come first");
  if (nrhs < 0 || (nrhs > 0 && (!d || !q))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  if (nrhs == 0) return TW_OK;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int nq = c->Nq * c->Nt, n = c->Nd * c->Nt;
  k_qoi_apply<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, (cudaStream_t)stream>>>(c->Qmap, d, q, nq, n, nrhs);
  count_launches(1);
  TW_CUDA(c, cudaGetLastError());
  return TW_OK;
}

tw_status tw_qoi_variance(tw_ctx *c, double *var, void *stream) {
  if (!c || !var) return TW_ERR_ARG;
  if (!c->have_qoi) return twh::fail(c, TW_ERR_STATE, "tw_qoi_build must come first");
  TW_CUDA(c, cudaSetDevice(c->dev));
  TW_CUDA(c, cudaMemcpyAsync(var, c->qvar, (size_t)c->Nq * c->Nt * sizeof(double),
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return TW_OK;
}

tw_status tw_qoi_covariance(tw_ctx *c, double *cov, void *stream) {
  if (!c || !cov) return TW_ERR_ARG;
  if (!c->have_qoi) return twh::fail(c, TW_ERR_STATE, "tw_qoi_build must come first");
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int nq = c->Nq * c->Nt, n = c->Nd * c->Nt;
  dim3 grid((nq + 63) / 64, (nq + 63) / 64);
  k_qoi_cov<<<grid, 256, 0, (cudaStream_t)stream>>>(c->Cqq, c->Wmap, c->Qmap, cov, nq, n);
  count_launches(1);
  TW_CUDA(c, cudaGetLastError());
  return TW_OK;
}

}  // extern "C"
