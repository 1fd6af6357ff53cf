// tw_batch.cu -- batches of right-hand sides with per-RHS observation windows.
//
// Phase 4 serves many events and posterior samples at once; with B
// right-hand sides the online path becomes
//   batched triangular solves  Z = L^-1 D,  Y = L^-T Z      (trsm.cu)
//   batched time FFTs, per-frequency products F^(w)^H Y^(w) (gemm.cu),
//   inverse FFTs and the prior filter                         (fft.cu)
// with every factor block and operator entry read once per column slice
// rather than once per right-hand side.  Windows live in device memory, so
// the calls below neither allocate nor synchronise and can be captured into
// one CUDA graph that is relaunched with new data and windows.
#include <algorithm>

#include "ctx.h"
#include "dense_api.h"

using namespace tw;

namespace {

// r[i] = d[i] - a[i] - sigma z[i] over B * n entries
// r may be a (in place): each thread reads and writes only its own entry
__global__ void k_sample_rhs_b(const double *d, const double *a, const double *z, double sigma, double *r,
                               long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = d[i] - a[i] - sigma * z[i];
}

// windows from a host array into device memory (stream-ordered copy of a
// pageable buffer: the host array may be reused once the call returns)
tw_status upload_windows(tw_ctx *c, const int *nt_window, int nrhs, cudaStream_t s) {
  std::vector<int> w(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    w[r] = nt_window ? nt_window[r] : c->Nt;
    if (w[r] < 1 || w[r] > c->Nt) return twh::fail(c, TW_ERR_ARG, "window must be in [1, Nt]");
  }
  TW_CUDA(c, cudaMemcpyAsync(c->lane.win_dev, w.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
  return TW_OK;
}

// lanes per right-hand side of the batched forward product, fixed per
// reservation (a column's sum order must not depend on its batch)
int fwd_lpb(const tw_lane &L) { return L.fwd_lpb; }

tw_status check_batch(tw_ctx *c, tw_prec prec, int nrhs, const int *win) {
  if (prec < 0 || prec > 2 || !c->op[TW_MAP_F][prec])
    return twh::fail(c, TW_ERR_ARG, "requested precision was not kept at tw_create");
  if (c->lane.bmax <= 0) return twh::fail(c, TW_ERR_STATE, "tw_reserve_batch must come first");
  if (nrhs > c->lane.bmax) return twh::fail(c, TW_ERR_ARG, "more right-hand sides than reserved");
  if (nrhs > 0 && !win) return twh::fail(c, TW_ERR_ARG, "windows (device array) required");
  if (!c->inv_dd || !c->have64)
    return twh::fail(c, TW_ERR_STATE, "batched solves need the FP64 factor (tw_factor_K)");
  return TW_OK;
}

}  // namespace

namespace twb {

// q = F_q m for B right-hand sides; rows t >= win[b] of m are taken as zero
// spec_ready: m's spectrum is already in L.bxh (the fused transform of infer_core)
tw_status forecast_core(tw_ctx *c, tw_lane &L, tw_prec prec, int B, const int *win, const double *m,
                        double *q, cudaStream_t s, bool spec_ready) {
  const int Nt = c->Nt, Nm = c->Nm, Nf = c->Nf, Nq = c->Nq;
  const void *Aq = c->op[TW_MAP_FQ][prec];
  const BatchArg ba_m{B, (long)Nt * Nm, (long)Nf * Nm, 0, win};
  const BatchArg ba_q{B, (long)Nf * Nq, (long)Nt * Nq, 0, nullptr};
  if (prec == TW_PREC_FP64) {
    if (!spec_ready) {
      twh::Phase p(c, TW_PH_RFFT_PARAM, s);
      TW_CUDA(c, launch_rfft_time_dd(m, 0, Nm, Nt, (cdd *)L.bxh, Nm, Nm, c->plT, c->twT, c->twL, s, ba_m));
    }
    { twh::Phase p(c, TW_PH_GEMV_FWD, s);
      TW_CUDA(c, launch_gemm_fwd_dd(Aq, (const cdd *)L.bxh, (long)Nf * Nm, (cdd *)L.bpart,
                                    (cdd *)L.byh, (long)Nf * Nq, Nf, Nq, Nm, B, s, fwd_lpb(L))); }
    { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
      TW_CUDA(c, launch_irfft_time_dd((const cdd *)L.byh, Nq, q, 0, Nq, Nq, Nt, c->plT, c->twT, c->twL, s, ba_q)); }
  } else {
    if (!spec_ready) {
      twh::Phase p(c, TW_PH_RFFT_PARAM, s);
      TW_CUDA(c, launch_rfft_time_f(m, 0, Nm, Nt, (cf *)L.bxh, Nm, Nm, c->plT, c->twTf, c->twLf, s, ba_m));
    }
    { twh::Phase p(c, TW_PH_GEMV_FWD, s);
      TW_CUDA(c, launch_gemm_fwd_f(Aq, (int)prec, (const cf *)L.bxh, (long)Nf * Nm, (cf *)L.bpart,
                                   (cf *)L.byh, (long)Nf * Nq, Nf, Nq, Nm, B, s, fwd_lpb(L))); }
    { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
      TW_CUDA(c, launch_irfft_time_f((const cf *)L.byh, Nq, q, 0, Nq, Nq, Nt, c->plT, c->twTf, c->twLf, s, ba_q)); }
  }
  return TW_OK;
}

// m = Gamma_pr F'^T K'^{-1} d' per right-hand side (window win[b]); rhs
// column b at rhs + b * rhs_bstride (FP64, [Nt][Nd]); q = F_q m if q != NULL
tw_status infer_core(tw_ctx *c, tw_lane &L, tw_prec prec, int B, const int *win, const double *rhs,
                     long rhs_bstride, double *m, double *q, cudaStream_t s) {
  const int Nd = c->Nd, Nt = c->Nt, Nm = c->Nm, Nf = c->Nf;
  const long np = c->n_pad;
  // with G^ = F^ C kept the adjoint gives m directly (no prior filter)
  const bool useG = c->opG[prec] != nullptr;
  const void *A = useG ? c->opG[prec] : c->op[TW_MAP_F][prec];
  int *prog_f = L.trsm_prog, *prog_b = L.trsm_prog + trsm_prog_ints(L.bmax);
  const BatchArg ba_y{B, np, (long)Nf * Nd, 0, win};
  const BatchArg ba_x{B, (long)Nf * Nm, (long)Nt * Nm, 0, win};
  // with G^ (no prior after the inverse transform) and a forecast requested,
  // the inverse transform of x^ and the forecast's forward transform of m
  // run as one kernel (as tw_infer_forecast does for one right-hand side)
  const bool fuse = q != nullptr && useG;
  const BatchArg ba_xf{B, (long)Nf * Nm, (long)Nt * Nm, (long)Nf * Nm, win};
  const BatchArg ba_p{B, (long)Nt * Nm, (long)Nt * Nm, (long)((Nt + 1) / 2) * Nm, win};
  if (prec == TW_PREC_FP64) {
    // double-float sweeps with the single-vector solve's pre-multiplied
    // blocks (FP64 products rounded to float pairs); y as float pairs in the
    // lane's 8-byte solve buffers
    dd *bz = reinterpret_cast<dd *>(L.bz), *by = reinterpret_cast<dd *>(L.by);
    { twh::Phase p(c, TW_PH_TRSV_FWD, s);
      TW_CUDA(c, launch_trsm_dd_scaled(c->Lfs, c->inv_dd, rhs, 0, rhs_bstride, bz, np, win, Nd, Nt, B,
                                       c->NB, prog_f, true, c->d_err, c->abort_flag, s)); }
    { twh::Phase p(c, TW_PH_TRSV_BWD, s);
      TW_CUDA(c, launch_trsm_dd_scaled(c->Lbs, c->inv_dd, bz, 1, np, by, np, win, Nd, Nt, B, c->NB,
                                       prog_b, false, c->d_err, c->abort_flag, s)); }
    { twh::Phase p(c, TW_PH_RFFT_DATA, s);
      TW_CUDA(c, launch_rfft_time_dd(by, 1, Nd, Nt, (cdd *)L.byh, Nd, Nd, c->plT, c->twT, c->twL, s, ba_y)); }
    { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
      TW_CUDA(c, launch_gemm_adj_dd(A, (const cdd *)L.byh, (long)Nf * Nd, (cdd *)L.bxh, (long)Nf * Nm,
                                    Nf, Nd, Nm, B, s, L.adj_rw)); }
    { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
      if (fuse)   // m, then m's spectrum in place of x^ (each CTA owns its columns)
        TW_CUDA(c, launch_irfft_rfft_time_dd((const cdd *)L.bxh, Nm, m, 0, Nm, (cdd *)L.bxh, Nm, Nm, Nt,
                                             c->plT, c->twT, c->twL, s, ba_xf));
      else
        TW_CUDA(c, launch_irfft_time_dd((const cdd *)L.bxh, Nm, m, 0, Nm, Nm, Nt, c->plT, c->twT, c->twL, s, ba_x)); }
    if (!useG) {
      twh::Phase p(c, TW_PH_PRIOR, s);
      TW_CUDA(c, launch_prior_dd(m, 0, m, 0, Nt, c->Nx, c->Ny, (cdd *)L.bxh, c->lam1, c->plX, c->plY,
                                 c->twX, c->twY, s, ba_p, 0));
    }
  } else {
    // the same double-float sweeps as the FP64 path
    { twh::Phase p(c, TW_PH_TRSV_FWD, s);
      TW_CUDA(c, launch_trsm_dd_scaled(c->Lfs, c->inv_dd, rhs, 0, rhs_bstride, L.bzd, np, win, Nd, Nt, B,
                                       c->NB, prog_f, true, c->d_err, c->abort_flag, s)); }
    { twh::Phase p(c, TW_PH_TRSV_BWD, s);
      TW_CUDA(c, launch_trsm_dd_scaled(c->Lbs, c->inv_dd, L.bzd, 1, np, L.byd, np, win, Nd, Nt, B, c->NB,
                                       prog_b, false, c->d_err, c->abort_flag, s)); }
    // double-float data spectra; the product on the tensor cores with both
    // sides cut into exact fixed-point slices: F^T y cancels (y is large
    // against m), so its sum has to be formed far below FP32 rounding
    { twh::Phase p(c, TW_PH_RFFT_DATA, s);
      TW_CUDA(c, launch_rfft_time_dd(L.byd, 1, Nd, Nt, (cdd *)L.byh, Nd, Nd, c->plT, c->twT, c->twL, s, ba_y)); }
    { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
      const int8_t *ea = useG ? c->eaG[prec] : c->ea[TW_MAP_F][prec];
      TW_CUDA(c, launch_gemm_adj_sl(A, (int)prec, ea, (const cdd *)L.byh, (long)Nf * Nd, (cf *)L.bxh,
                                    (long)Nf * Nm, Nf, Nd, Nm, B, L.sl_tile, L.bsl_ws, L.bsl_ws_n,
                                    L.bsl_eb, L.bsl_eb_n, c->d_err, s)); }
    { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
      if (fuse)
        TW_CUDA(c, launch_irfft_rfft_time_f((const cf *)L.bxh, Nm, m, 0, Nm, (cf *)L.bxh, Nm, Nm, Nt, c->plT,
                                            c->twTf, c->twLf, s, ba_xf));
      else
        TW_CUDA(c, launch_irfft_time_f((const cf *)L.bxh, Nm, m, 0, Nm, Nm, Nt, c->plT, c->twTf, c->twLf, s, ba_x)); }
    if (!useG) {
      twh::Phase p(c, TW_PH_PRIOR, s);
      TW_CUDA(c, launch_prior_f(m, 0, m, 0, Nt, c->Nx, c->Ny, (cf *)L.bxh, c->lam1f, c->plX, c->plY,
                                c->twXf, c->twYf, s, ba_p, 0));
    }
  }
  if (q) return forecast_core(c, L, prec, B, win, m, q, s, fuse);
  return TW_OK;
}

// s = m_pr + Gamma_pr F'^T K'^{-1} (d' - F' m_pr - sigma z_n), m_pr = Gamma_pr^{1/2} z_m
tw_status sample_core(tw_ctx *c, tw_lane &L, tw_prec prec, int B, const int *win, const double *d,
                      const double *z_m, const double *z_n, double sigma, double *samples,
                      cudaStream_t s) {
  const int Nd = c->Nd, Nt = c->Nt, Nm = c->Nm, Nf = c->Nf;
  const void *A = c->op[TW_MAP_F][prec];
  const BatchArg ba_full{B, (long)Nt * Nm, (long)Nt * Nm, (long)((Nt + 1) / 2) * Nm, nullptr};
  const BatchArg ba_m{B, (long)Nt * Nm, (long)Nf * Nm, 0, win};
  const BatchArg ba_d{B, (long)Nf * Nd, (long)Nt * Nd, 0, win};
  const bool f64 = prec == TW_PREC_FP64;
  // m_pr into the output
  { twh::Phase p(c, TW_PH_PRIOR, s);
    if (f64) TW_CUDA(c, launch_prior_dd(z_m, 0, samples, 0, Nt, c->Nx, c->Ny, (cdd *)L.bxh, c->lamh,
                                        c->plX, c->plY, c->twX, c->twY, s, ba_full, 0));
    else TW_CUDA(c, launch_prior_f(z_m, 0, samples, 0, Nt, c->Nx, c->Ny, (cf *)L.bxh, c->lamhf,
                                   c->plX, c->plY, c->twXf, c->twYf, s, ba_full, 0)); }
  // a = F' m_pr (the leading window blocks depend on m_pr's leading blocks only)
  if (f64) {
    { twh::Phase p(c, TW_PH_RFFT_PARAM, s);
      TW_CUDA(c, launch_rfft_time_dd(samples, 0, Nm, Nt, (cdd *)L.bxh, Nm, Nm, c->plT, c->twT, c->twL, s, ba_m)); }
    { twh::Phase p(c, TW_PH_GEMV_FWD, s);
      TW_CUDA(c, launch_gemm_fwd_dd(A, (const cdd *)L.bxh, (long)Nf * Nm, (cdd *)L.bpart, (cdd *)L.byh,
                                    (long)Nf * Nd, Nf, Nd, Nm, B, s, fwd_lpb(L))); }
    { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
      TW_CUDA(c, launch_irfft_time_dd((const cdd *)L.byh, Nd, L.brd, 0, Nd, Nd, Nt, c->plT, c->twT, c->twL, s, ba_d)); }
  } else {
    { twh::Phase p(c, TW_PH_RFFT_PARAM, s);
      TW_CUDA(c, launch_rfft_time_f(samples, 0, Nm, Nt, (cf *)L.bxh, Nm, Nm, c->plT, c->twTf, c->twLf, s, ba_m)); }
    { twh::Phase p(c, TW_PH_GEMV_FWD, s);
      TW_CUDA(c, launch_gemm_fwd_f(A, (int)prec, (const cf *)L.bxh, (long)Nf * Nm, (cf *)L.bpart,
                                   (cf *)L.byh, (long)Nf * Nd, Nf, Nd, Nm, B, s, fwd_lpb(L))); }
    { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
      TW_CUDA(c, launch_irfft_time_f((const cf *)L.byh, Nd, L.brd, 0, Nd, Nd, Nt, c->plT, c->twTf, c->twLf, s, ba_d)); }
  }
  const long nd = (long)B * Nt * Nd;
  k_sample_rhs_b<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(d, L.brd, z_n, sigma, L.brd, nd);
  count_launches(1);
  TW_CUDA(c, cudaGetLastError());
  tw_status st = infer_core(c, L, prec, B, win, L.brd, (long)Nt * Nd, samples, nullptr, s);
  if (st != TW_OK) return st;
  // add m_pr back (recomputed: no second parameter-sized buffer is needed)
  twh::Phase p(c, TW_PH_PRIOR, s);
  if (f64) TW_CUDA(c, launch_prior_dd(z_m, 0, samples, 0, Nt, c->Nx, c->Ny, (cdd *)L.bxh, c->lamh,
                                      c->plX, c->plY, c->twX, c->twY, s, ba_full, 1));
  else TW_CUDA(c, launch_prior_f(z_m, 0, samples, 0, Nt, c->Nx, c->Ny, (cf *)L.bxh, c->lamhf,
                                 c->plX, c->plY, c->twXf, c->twYf, s, ba_full, 1));
  return TW_OK;
}

size_t lane_bytes(const tw_ctx *c, int bmax) {
  const size_t B = bmax, np = c->n_pad, Nt = c->Nt, Nf = c->Nf, Nm = c->Nm, R = c->Rmax;
  const bool mixed = c->op[TW_MAP_F][TW_PREC_C64] || c->op[TW_MAP_F][TW_PREC_BF16X2];
  size_t b = B * sizeof(int) + 2 * (size_t)trsm_prog_ints(bmax) * sizeof(int) + 2 * B * np * sizeof(double) +
             B * Nt * c->Nd * sizeof(double) + B * Nf * R * sizeof(cdd) + B * Nf * Nm * sizeof(cdd) +
             B * Nf * (size_t)gemm_fwd_nchunk(c->Nm) * R * sizeof(cdd);
  if (mixed) {
    const int cols = (bmax + 7) / 8 * 8 + 80;
    b += 2 * B * np * sizeof(dd) + sl_ws_bytes(c->Nf, c->Rmax, cols) + sl_eb_bytes(c->Nf, cols);
  }
  return b;
}

void free_lane(tw_ctx *c, tw_lane &L) {
  void **bufs[] = {(void **)&L.win_dev, (void **)&L.trsm_prog, (void **)&L.bz, (void **)&L.by,
                   (void **)&L.bzd, (void **)&L.byd, (void **)&L.brd, &L.byh, &L.bxh, &L.bpart,
                   &L.bsl_ws, (void **)&L.bsl_eb};
  for (void **b : bufs) { twh::dfree(c, *b); *b = nullptr; }
  L.bmax = 0;
  L.bytes = 0;
}

tw_status alloc_lane(tw_ctx *c, tw_lane &L, int bmax) {
  free_lane(c, L);
  const size_t B = bmax, np = c->n_pad, Nt = c->Nt, Nf = c->Nf, Nm = c->Nm, R = c->Rmax;
  const bool mixed = c->op[TW_MAP_F][TW_PREC_C64] || c->op[TW_MAP_F][TW_PREC_BF16X2];
  bool ok = true;
  auto take = [&](size_t bytes) -> void * {
    void *p = twh::dalloc(c, bytes);
    ok = ok && p;
    return p;
  };
  L.win_dev = (int *)take(B * sizeof(int));
  L.trsm_prog = (int *)take(2 * (size_t)trsm_prog_ints(bmax) * sizeof(int));
  L.bz = (double *)take(B * np * sizeof(double));
  L.by = (double *)take(B * np * sizeof(double));
  L.brd = (double *)take(B * Nt * c->Nd * sizeof(double));
  L.byh = take(B * Nf * R * sizeof(cdd));
  L.bxh = take(B * Nf * Nm * sizeof(cdd));   // >= B * ceil(Nt/2) * Nm: also the prior's work
  L.bpart = take(B * Nf * (size_t)gemm_fwd_nchunk(c->Nm) * R * sizeof(cdd));
  if (mixed) {
    L.bzd = (dd *)take(B * np * sizeof(dd));
    L.byd = (dd *)take(B * np * sizeof(dd));
    // data-side slices of the tensor-core adjoint, for any tile P <= 80:
    // ceil(bmax / P) P < bmax + 80 columns
    L.sl_tile = sl_pick_tile(bmax);
    const int cols = (bmax + 7) / 8 * 8 + 80;
    L.bsl_ws_n = sl_ws_bytes(c->Nf, c->Rmax, cols);
    L.bsl_eb_n = sl_eb_bytes(c->Nf, cols);
    L.bsl_ws = take(L.bsl_ws_n);
    L.bsl_eb = (int *)take(L.bsl_eb_n);
  }
  if (!ok) {
    free_lane(c, L);
    return twh::fail(c, TW_ERR_OOM, "batch workspaces");
  }
  L.bmax = bmax;
  L.adj_rw = 0;
  L.fwd_lpb = bmax <= 16 ? 2 : 1;      // defaults until measured
  L.bytes = lane_bytes(c, bmax);
  TW_CUDA(c, cudaMemset(L.win_dev, 0, B * sizeof(int)));
  return TW_OK;
}

}  // namespace twb

namespace {

void free_batch(tw_ctx *c) {
  twb::free_lane(c, c->lane);
  twh::dfree(c, c->inv_dd);
  c->inv_dd = nullptr;
}

}  // namespace

tw_status twh::refresh_dd_factor(tw_ctx *c, cudaStream_t s) {
  if (!c->have64) return TW_OK;
  if (c->inv_dd) TW_CUDA(c, launch_double_to_dd(c->inv64, c->inv_dd, (size_t)c->NB * NB_ * NB_, s));
  TW_CUDA(c, cudaStreamSynchronize(s));
  return TW_OK;
}

extern "C" {

tw_status tw_reserve_batch(tw_ctx *c, int bmax) {
  if (!c) return TW_ERR_ARG;
  if (bmax < 0) return twh::fail(c, TW_ERR_ARG, "bmax must be >= 0");
  if (!c->have64) return twh::fail(c, TW_ERR_STATE, "tw_factor_K (FP64 factor) must come first");
  TW_CUDA(c, cudaSetDevice(c->dev));
  TW_CUDA(c, cudaDeviceSynchronize());
  free_batch(c);
  if (bmax == 0) return TW_OK;
  // float-pair diagonal-block inverses for the batched solves (their blocks
  // are the single-vector solve's pre-multiplied float-pair factor)
  c->inv_dd = (dd *)twh::dalloc(c, (size_t)c->NB * NB_ * NB_ * sizeof(dd));
  if (!c->inv_dd) {
    free_batch(c);
    return twh::fail(c, TW_ERR_OOM, "batch workspaces");
  }
  tw_status st = twb::alloc_lane(c, c->lane, bmax);
  if (st != TW_OK) {
    free_batch(c);
    return st;
  }
  st = twh::refresh_dd_factor(c, 0);
  if (st != TW_OK) return st;
  return twb::autotune_lane(c, c->lane);
}

int tw_batch_capacity(const tw_ctx *c) { return c ? c->lane.bmax : -1; }

tw_status tw_infer_batch(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window_dev,
                         const double *d, double *m, double *q, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nrhs < 0 || (nrhs > 0 && (!d || !m))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  tw_status st = check_batch(c, prec, nrhs, nt_window_dev);
  if (st != TW_OK || nrhs == 0) return st;
  TW_CUDA(c, cudaSetDevice(c->dev));
  return twb::infer_core(c, c->lane, prec, nrhs, nt_window_dev, d, (long)c->Nt * c->Nd, m, q, (cudaStream_t)stream);
}

tw_status tw_sample_posterior_batch(tw_ctx *c, tw_prec prec, int ns, const int *nt_window_dev,
                                    const double *d, const double *z_m, const double *z_n,
                                    double sigma, double *samples, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (ns < 0 || (ns > 0 && (!d || !z_m || !z_n || !samples)))
    return twh::fail(c, TW_ERR_ARG, "bad sample arguments");
  if (!(sigma >= 0.0)) return twh::fail(c, TW_ERR_ARG, "sigma must be >= 0");
  tw_status st = check_batch(c, prec, ns, nt_window_dev);
  if (st != TW_OK || ns == 0) return st;
  TW_CUDA(c, cudaSetDevice(c->dev));
  return twb::sample_core(c, c->lane, prec, ns, nt_window_dev, d, z_m, z_n, sigma, samples, (cudaStream_t)stream);
}

tw_status tw_forecast_batch(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window_dev,
                            const double *m, double *q, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nrhs < 0 || (nrhs > 0 && (!m || !q))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  if (prec < 0 || prec > 2 || !c->op[TW_MAP_FQ][prec])
    return twh::fail(c, TW_ERR_ARG, "requested precision was not kept at tw_create");
  if (c->lane.bmax <= 0) return twh::fail(c, TW_ERR_STATE, "tw_reserve_batch must come first");
  if (nrhs > c->lane.bmax) return twh::fail(c, TW_ERR_ARG, "more right-hand sides than reserved");
  if (nrhs == 0) return TW_OK;
  TW_CUDA(c, cudaSetDevice(c->dev));
  return twb::forecast_core(c, c->lane, prec, nrhs, nt_window_dev, m, q, (cudaStream_t)stream, false);
}

// ---- CUDA graphs of batched calls
struct tw_graph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
};

tw_status tw_capture_begin(tw_ctx *c, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (!stream) return twh::fail(c, TW_ERR_ARG, "capture needs a created stream (not the default)");
  TW_CUDA(c, cudaSetDevice(c->dev));
  TW_CUDA(c, cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeRelaxed));
  return TW_OK;
}

tw_status tw_capture_end(tw_ctx *c, void *stream, tw_graph **out) {
  if (!c || !out) return TW_ERR_ARG;
  *out = nullptr;
  cudaGraph_t g = nullptr;
  TW_CUDA(c, cudaStreamEndCapture((cudaStream_t)stream, &g));
  tw_graph *h = new tw_graph;
  h->g = g;
  cudaError_t e = cudaGraphInstantiate(&h->x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    delete h;
    return twh::cuda_fail(c, e, "cudaGraphInstantiate");
  }
  *out = h;
  return TW_OK;
}

tw_status tw_graph_launch(tw_graph *h, void *stream) {
  if (!h || !h->x) return TW_ERR_ARG;
  return cudaGraphLaunch(h->x, (cudaStream_t)stream) == cudaSuccess ? TW_OK : TW_ERR_CUDA;
}

int tw_graph_kernel_count(const tw_graph *h) {
  if (!h || !h->g) return -1;
  size_t n = 0;
  if (cudaGraphGetNodes(h->g, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(h->g, nodes.data(), &n) != cudaSuccess) return -1;
  int k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

void tw_graph_destroy(tw_graph *h) {
  if (!h) return;
  if (h->x) cudaGraphExecDestroy(h->x);
  if (h->g) cudaGraphDestroy(h->g);
  delete h;
}

}  // extern "C"

// host-window entry points route here when a batch is reserved
namespace twb {

tw_status infer_host_windows(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window,
                             const double *d, double *m, cudaStream_t s) {
  for (int r0 = 0; r0 < nrhs; r0 += c->lane.bmax) {
    const int nb = std::min(c->lane.bmax, nrhs - r0);
    tw_status st = upload_windows(c, nt_window ? nt_window + r0 : nullptr, nb, s);
    if (st != TW_OK) return st;
    st = infer_core(c, c->lane, prec, nb, c->lane.win_dev, d + (size_t)r0 * c->Nt * c->Nd, (long)c->Nt * c->Nd,
                    m + (size_t)r0 * c->Nt * c->Nm, nullptr, s);
    if (st != TW_OK) return st;
  }
  return TW_OK;
}

tw_status sample_host_windows(tw_ctx *c, int ns, const int *nt_window, const double *d,
                              const double *z_m, const double *z_n, double sigma, double *samples,
                              cudaStream_t s) {
  const size_t pm = (size_t)c->Nt * c->Nm, pd = (size_t)c->Nt * c->Nd;
  for (int k0 = 0; k0 < ns; k0 += c->lane.bmax) {
    const int nb = std::min(c->lane.bmax, ns - k0);
    tw_status st = upload_windows(c, nt_window ? nt_window + k0 : nullptr, nb, s);
    if (st != TW_OK) return st;
    st = sample_core(c, c->lane, TW_PREC_FP64, nb, c->lane.win_dev, d + k0 * pd, z_m + k0 * pm, z_n + k0 * pd,
                     sigma, samples + k0 * pm, s);
    if (st != TW_OK) return st;
  }
  return TW_OK;
}

tw_status forecast_full(tw_ctx *c, tw_prec prec, int nrhs, const double *m, double *q,
                        cudaStream_t s) {
  const size_t pm = (size_t)c->Nt * c->Nm, pq = (size_t)c->Nt * c->Nq;
  for (int r0 = 0; r0 < nrhs; r0 += c->lane.bmax) {
    const int nb = std::min(c->lane.bmax, nrhs - r0);
    tw_status st = forecast_core(c, c->lane, prec, nb, nullptr, m + r0 * pm, q + r0 * pq, s, false);
    if (st != TW_OK) return st;
  }
  return TW_OK;
}

}  // namespace twb
