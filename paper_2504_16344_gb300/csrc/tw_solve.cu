// tw_solve.cu -- K formation and factorisation, posterior mean, forecast.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>

#include "ctx.h"
#include "dense_api.h"

using namespace tw;

namespace {

tw_status ensure_solve_workspace(tw_ctx *c) {
  if (c->vz) return TW_OK;
  const size_t np = c->n_pad;
  c->vz = (dd *)twh::dalloc(c, np * sizeof(dd));
  c->vy = (dd *)twh::dalloc(c, np * sizeof(dd));
  c->vr = (dd *)twh::dalloc(c, np * sizeof(dd));
  c->zd = (double *)twh::dalloc(c, np * sizeof(double));
  c->yd = (double *)twh::dalloc(c, np * sizeof(double));
  c->rd = (double *)twh::dalloc(c, np * sizeof(double));
  c->ad = (double *)twh::dalloc(c, np * sizeof(double));
  c->fz = (float *)twh::dalloc(c, np * sizeof(float));
  c->fy = (float *)twh::dalloc(c, np * sizeof(float));
  c->counter = (int *)twh::dalloc(c, 4 * sizeof(int));
  c->abort_flag = (int *)twh::dalloc(c, sizeof(int));
  c->d_norm = (double *)twh::dalloc(c, 2 * sizeof(double));
  if (!c->vz || !c->vy || !c->vr || !c->zd || !c->yd || !c->rd || !c->ad || !c->fz || !c->fy || !c->counter || !c->abort_flag || !c->d_norm)
    return twh::fail(c, TW_ERR_OOM, "solve workspace");
  TW_CUDA(c, cudaMemset(c->vz, 0, np * sizeof(dd)));
  TW_CUDA(c, cudaMemset(c->vy, 0, np * sizeof(dd)));
  TW_CUDA(c, cudaMemset(c->counter, 0, 4 * sizeof(int)));
  TW_CUDA(c, cudaMemset(c->abort_flag, 0, sizeof(int)));
  return TW_OK;
}

// y = K^{-1} b for the leading nrows with the FP64 factor: block-scaled
// factor as float pairs, double-float products (2^-48 rounding; at the test
// cases' condition numbers, up to 2.3e6, it moves m by under 1e-12)
// b: double (kind 0) or dd (kind 1)
tw_status solve64(tw_ctx *c, const void *b, int kind, int nrows, double *y, cudaStream_t s) {
  const int NBw = (nrows + NB_ - 1) / NB_;
  Trsv64Args a{};
  a.Lf = c->Lfs; a.Lb = c->Lbs; a.Linv = c->inv64; a.bands = c->bands; a.NB = c->NB;
  a.nrows = nrows; a.NBw = NBw; a.tasks = c->tasks; a.ntasks = c->task_prefix[NBw];
  a.part = c->tpart; a.maxk = c->tmaxk; a.cnt = c->tcnt; a.wbuf = c->wbufx;
  a.outx = c->zx;
  a.err = c->d_err; a.abort_flag = c->abort_flag;
  { twh::Phase p(c, TW_PH_TRSV_FWD, s);
    a.rhs = b; a.rhs_kind = kind; a.out = c->zd; a.prog = c->counter;
    TW_CUDA(c, launch_trsv64(a, true, s)); }
  twh::Phase p(c, TW_PH_TRSV_BWD, s);
  a.rhs = c->zd; a.rhs_kind = 0; a.out = y; a.prog = c->counter + 2;
  TW_CUDA(c, launch_trsv64(a, false, s));
  return TW_OK;
}

// float solve with the FP32 factor: y32 = K32^{-1} b
tw_status solve32(tw_ctx *c, const void *b, int kind, int nrows, float *y, cudaStream_t s) {
  const int NBw = (nrows + NB_ - 1) / NB_;
  { twh::Phase p(c, TW_PH_TRSV_FWD, s);
    TW_CUDA(c, launch_trsv_f(c->Lp32, c->inv32, c->chF32, b, kind, c->fz, nrows, NBw, c->counter,
                             true, c->d_err, c->abort_flag, s)); }
  twh::Phase p(c, TW_PH_TRSV_BWD, s);
  TW_CUDA(c, launch_trsv_f(c->Lp32, c->inv32, c->chB32, c->fz, 2, y, nrows, NBw, c->counter + 2,
                           false, c->d_err, c->abort_flag, s));
  return TW_OK;
}

// After the FP64 factor (Lp64, inv64) is in place: the solves' chain blocks,
// the single-vector solve's block-scaled factor and task table.
tw_status finish_factor64(tw_ctx *c, cudaStream_t s) {
  twh::Phase ph(c, TW_PH_SOLVE_SETUP, s);
  const size_t nblk = (size_t)c->NB * (c->NB + 1) / 2;
  const size_t blk = (size_t)NB_ * NB_;
  const size_t np = c->n_pad;
  if (!c->chF64) c->chF64 = (double *)twh::dalloc(c, (size_t)c->NB * blk * sizeof(double));
  if (!c->chB64) c->chB64 = (double *)twh::dalloc(c, (size_t)c->NB * blk * sizeof(double));
  if (!c->chF64 || !c->chB64) return twh::fail(c, TW_ERR_OOM, "chain blocks");
  TW_CUDA(c, launch_chain_blocks_d(c->Lp64, c->inv64, c->chF64, c->chB64, c->NB, s));
  std::vector<int> tab;
  trsv64_task_table(c->NB, tab, c->task_prefix);
  c->tmaxk = trsv64_max_tasks_per_row(c->NB);
  auto need = [&](void *&p, size_t bytes) { if (!p) p = twh::dalloc(c, bytes); return p != nullptr; };
  bool ok = need((void *&)c->Lfs, nblk * blk * sizeof(dd)) &&
            need((void *&)c->Lbs, nblk * blk * sizeof(dd)) &&
            need((void *&)c->bands, (size_t)2 * trsv64_chain_deps() * c->NB * blk * sizeof(dd)) &&
            need((void *&)c->tasks, tab.size() / 2 * sizeof(int2)) &&
            need((void *&)c->tpart, (size_t)c->NB * c->tmaxk * NB_ * sizeof(dd)) &&
            need((void *&)c->tcnt, (size_t)c->NB * sizeof(int)) &&
            need((void *&)c->wbufx, np * sizeof(dd)) &&
            need((void *&)c->zx, np * sizeof(dd));
  if (!ok) return twh::fail(c, TW_ERR_OOM, "single-vector solve buffers");
  TW_CUDA(c, cudaMemcpyAsync(c->tasks, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  TW_CUDA(c, launch_trsv64_setup(c->Lp64, c->inv64, c->Lfs, c->Lbs, c->bands, c->NB, s));
  TW_CUDA(c, cudaStreamSynchronize(s));
  tw_status cs = tw_check(c, s);
  if (cs != TW_OK) return cs;
  c->have64 = true;
  return TW_OK;
}

// Phase 2's G* = Gamma_pr F*: G^ = F^ C per frequency, FP64 filter on the
// FP64 storage, then converted to the other kept formats (TW_KEEP_G)
tw_status form_gstar(tw_ctx *c, cudaStream_t s) {
  if (!(c->keep & TW_KEEP_G) || !c->op[TW_MAP_F][TW_PREC_FP64]) return TW_OK;
  twh::Phase ph(c, TW_PH_FORM_GSTAR, s);
  const size_t per_w = (size_t)c->Nd * c->Nm;
  // FP64 and complex64 only: bf16 hi+lo storage of G^ rounds at 2^-18 and
  // that rounding reaches m unsmoothed (1.3e-5 .. 1.6e-5 measured); the
  // bf16x2 path keeps F^ and the FP32 prior filter
  for (int fmt = 0; fmt < 2; ++fmt) {
    if (!c->op[TW_MAP_F][fmt] || c->opG[fmt]) continue;
    c->opG[fmt] = twh::dalloc(c, (size_t)c->Nf * per_w * (fmt == 0 ? sizeof(cdd) : sizeof(cf)));
    if (!c->opG[fmt]) return twh::fail(c, TW_ERR_OOM, "G^ storage");
  }
  TW_CUDA(c, cudaMemcpyAsync(c->opG[0], c->op[TW_MAP_F][0], (size_t)c->Nf * per_w * sizeof(cdd),
                             cudaMemcpyDeviceToDevice, s));
  TW_CUDA(c, launch_prior_cfields_d((cdd *)c->opG[0], (long)c->Nf * c->Nd, c->Nx, c->Ny, (cd *)c->ws,
                                    (c->Nt + 1) / 2, c->lam1d, c->plX, c->plY, c->twXd, c->twYd, s));
  for (int fmt = 1; fmt < 2; ++fmt)
    if (c->opG[fmt]) {
      TW_CUDA(c, launch_convert_op((const cdd *)c->opG[0], (long)per_w, c->opG[fmt], fmt, (long)per_w,
                                   (long)per_w, c->Nf, s));
      if (!c->eaG[fmt]) {
        c->eaG[fmt] = (int8_t *)twh::dalloc(c, (size_t)c->Nf * c->Nm);
        if (!c->eaG[fmt]) return twh::fail(c, TW_ERR_OOM, "G^ row exponents");
      }
      TW_CUDA(c, launch_row_exp(c->opG[fmt], fmt, c->eaG[fmt], c->Nf, c->Nd, c->Nm, s));
    }
  TW_CUDA(c, cudaStreamSynchronize(s));
  return TW_OK;
}

// Phase-2 checkpoint: a fixed header, then the packed FP64 factor blocks and
// the inverses of its diagonal blocks
struct FactorHeader {
  char magic[8];
  int32_t Nd, Nt, Nx, Ny, NB, blk;
  uint64_t nblk;
  double sigma2, nu, ell, var, Lx, Ly;
  uint64_t col_hash;      // fingerprint of the block column of F that K was formed from
};
static_assert(sizeof(FactorHeader) == 96, "checkpoint header layout");
const char kFactorMagic[8] = {'T', 'W', 'L', 'F', 'A', 'C', '0', '2'};

size_t factor_payload(int NB) {
  const size_t nblk = (size_t)NB * (NB + 1) / 2;
  return (nblk + (size_t)NB) * NB_ * NB_ * sizeof(double);
}

}  // namespace

extern "C" {

tw_status tw_factor_K(tw_ctx *c, double noise_var, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (!(noise_var >= 0.0)) return twh::fail(c, TW_ERR_ARG, "noise variance must be >= 0");
  if (!c->prior_set) return twh::fail(c, TW_ERR_STATE, "tw_set_prior must come before tw_factor_K");
  for (char l : c->loaded[TW_MAP_F])
    if (!l) return twh::fail(c, TW_ERR_STATE, "block column of F not fully loaded");
  bool have_G = c->G != nullptr;
  for (char g : c->g_rows) have_G = have_G && g;
  if (!have_G && !c->op[TW_MAP_F][FMT_DD])
    return twh::fail(c, TW_ERR_STATE,
                     "without the FP64 operator, tw_set_prior must come before the block column of F");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int Nd = c->Nd, Nt = c->Nt, Nm = c->Nm;
  c->n = Nd * Nt;
  c->NB = (c->n + NB_ - 1) / NB_;
  c->n_pad = c->NB * NB_;
  c->sigma2 = noise_var;
  const long n = c->n, np = c->n_pad;
  const bool want64 = (c->keep & (TW_KEEP_FP64 | TW_KEEP_FACTOR64)) != 0;
  const bool want32 = (c->keep & (TW_KEEP_C64 | TW_KEEP_BF16X2)) != 0 && !(c->keep & TW_KEEP_FACTOR64);
  c->have64 = c->have32 = false;
  c->have_qoi = false;
  tw_status st = ensure_solve_workspace(c);
  if (st != TW_OK) return st;

  // G = Phi C^{1/2}, rows u*Nd + s.  Normally built in FP64 while the block
  // column was loaded (tw_set_prior first); otherwise Phi is recovered from
  // the stored operator by the inverse time FFT (K then carries ~1e-14
  // relative error from the double-float operator and filter).
  // K's formation is timed as one phase (a scope would not end at the packing)
  std::unique_ptr<twh::Phase> ph(new twh::Phase(c, TW_PH_FORM_K, s));
  dd *G = c->G;
  if (!have_G) {
    if (!G) G = (dd *)twh::dalloc(c, (size_t)n * Nm * sizeof(dd));
    if (!G) return twh::fail(c, TW_ERR_OOM, "G = Phi C^{1/2} buffer");
    const long ld = (long)Nd * Nm;
    TW_CUDA(c, launch_irfft_time_dd((const cdd *)c->op[TW_MAP_F][FMT_DD], ld, G, 1, ld, (int)ld, Nt,
                                    c->plT, c->twT, c->twL, s));
    const int chunk = 2 * ((Nt + 1) / 2);
    for (long r0 = 0; r0 < n; r0 += chunk) {
      const int nr = (int)std::min<long>(chunk, n - r0);
      dd *g = G + r0 * Nm;
      TW_CUDA(c, launch_prior_dd(g, 1, g, 1, nr, c->Nx, c->Ny, c->ws, c->lamh, c->plX, c->plY,
                                 c->twX, c->twY, s));
    }
  }
  c->G = nullptr;                       // consumed below
  std::fill(c->g_rows.begin(), c->g_rows.end(), 0);
  // P = G G^T, then K = sigma^2 I + block-diagonal prefix sums of P
  double *K = (double *)twh::dalloc(c, (size_t)np * np * sizeof(double));
  if (!K) { twh::dfree(c, G); return twh::fail(c, TW_ERR_OOM, "K buffer"); }
  TW_CUDA(c, cudaMemsetAsync(K, 0, (size_t)np * np * sizeof(double), s));
  {
    // P on the tensor cores from exact slices of G, one panel of up to 8192
    // grid points of slices at a time (as large as free memory allows)
    std::vector<int2> tl;
    syrk_tile_list((int)np, tl);
    const size_t per_atom = syrk_ws_bytes_per_atom((int)np);
    size_t free_b = 0, total_b = 0;
    TW_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
    const size_t margin = (size_t)2 << 30;
    const size_t avail = free_b > margin ? free_b - margin : 0;
    const size_t wsb = std::min(per_atom * 256, avail / per_atom * per_atom);
    int2 *dtl = (int2 *)twh::dalloc(c, tl.size() * sizeof(int2));
    int *eg = (int *)twh::dalloc(c, (size_t)syrk_exp_rows((int)np) * sizeof(int));
    uint8_t *ws = wsb >= per_atom * 4 ? (uint8_t *)twh::dalloc(c, wsb) : nullptr;
    if (!dtl || !eg || !ws) {
      twh::dfree(c, ws); twh::dfree(c, eg); twh::dfree(c, dtl); twh::dfree(c, K); twh::dfree(c, G);
      return twh::fail(c, TW_ERR_OOM, "slices of G for K's formation");
    }
    TW_CUDA(c, cudaMemcpyAsync(dtl, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    TW_CUDA(c, launch_form_P_tc(G, Nm, (int)n, Nm, K, np, (int)np, ws, wsb, eg, dtl, (int)tl.size(),
                                c->d_err, s));
    TW_CUDA(c, cudaStreamSynchronize(s));
    twh::dfree(c, ws);
    twh::dfree(c, eg);
    twh::dfree(c, dtl);
    tw_status cs = tw_check(c, s);
    if (cs != TW_OK) { twh::dfree(c, K); twh::dfree(c, G); return cs; }
  }
  twh::dfree(c, G);
  TW_CUDA(c, launch_K_from_P(K, np, Nd, Nt, (int)n, (int)np, noise_var, s));

  const size_t nblk = (size_t)c->NB * (c->NB + 1) / 2;
  const size_t blk = (size_t)NB_ * NB_;
  // K itself is kept (packed double-float blocks): refinement residuals,
  // tw_apply_K and residual certificates use it
  if (!c->Kp64) c->Kp64 = (dd *)twh::dalloc(c, nblk * blk * sizeof(dd));
  if (!c->Kp64) { twh::dfree(c, K); return twh::fail(c, TW_ERR_OOM, "packed K"); }
  TW_CUDA(c, launch_pack_d2dd(K, np, c->Kp64, c->NB, s));
  ph.reset();
  // mixed path: FP32 factor
  if (want32) {
    twh::Phase p32(c, TW_PH_CHOLESKY32, s);
    if (!c->Lp32) c->Lp32 = (float *)twh::dalloc(c, nblk * blk * sizeof(float));
    if (!c->inv32) c->inv32 = (float *)twh::dalloc(c, (size_t)c->NB * blk * sizeof(float));
    float *K32 = (float *)twh::dalloc(c, (size_t)np * np * sizeof(float));
    if (!c->Lp32 || !c->inv32 || !K32) {
      twh::dfree(c, K32);
      twh::dfree(c, K);
      return twh::fail(c, TW_ERR_OOM, "mixed-precision factor buffers");
    }
    // FP32 Cholesky; if it meets a non-positive pivot, add a small diagonal shift
    // (the refinement residual uses the unshifted FP64 K, so the solution is unchanged)
    c->shift32 = 0.0;
    for (int attempt = 0; attempt < 4; ++attempt) {
      TW_CUDA(c, cudaMemsetAsync(K32, 0, (size_t)np * np * sizeof(float), s));
      TW_CUDA(c, launch_lower_to_float(K, K32, np, c->NB, s));
      if (c->shift32 > 0.0) {
        // add the shift on the host-visible diagonal through a tiny kernel-free path
        std::vector<float> diag(np);
        TW_CUDA(c, cudaStreamSynchronize(s));
        TW_CUDA(c, cudaMemcpy2D(diag.data(), sizeof(float), K32, (np + 1) * sizeof(float),
                                sizeof(float), np, cudaMemcpyDeviceToHost));
        for (long i = 0; i < n; ++i) diag[i] += (float)c->shift32;
        TW_CUDA(c, cudaMemcpy2D(K32, (np + 1) * sizeof(float), diag.data(), sizeof(float),
                                sizeof(float), np, cudaMemcpyHostToDevice));
      }
      TW_CUDA(c, launch_cholesky_f(K32, np, c->NB, c->inv32, c->d_err, s));
      tw_status cs = tw_check(c, stream);
      if (cs == TW_OK) break;
      if (cs != TW_ERR_NOT_SPD || attempt == 3) { twh::dfree(c, K32); twh::dfree(c, K); return cs; }
      // shift relative to the largest diagonal entry (read back once)
      std::vector<double> dg(np);
      TW_CUDA(c, cudaMemcpy2D(dg.data(), sizeof(double), K, (np + 1) * sizeof(double),
                              sizeof(double), np, cudaMemcpyDeviceToHost));
      double dmax = 0.0;
      for (long i = 0; i < n; ++i) dmax = std::max(dmax, dg[i]);
      c->shift32 = (c->shift32 == 0.0) ? dmax * 1e-6 : c->shift32 * 10.0;
    }
    TW_CUDA(c, launch_pack_f(K32, np, c->Lp32, c->NB, s));
    if (!c->chF32) c->chF32 = (float *)twh::dalloc(c, (size_t)c->NB * blk * sizeof(float));
    if (!c->chB32) c->chB32 = (float *)twh::dalloc(c, (size_t)c->NB * blk * sizeof(float));
    if (!c->chF32 || !c->chB32) { twh::dfree(c, K32); twh::dfree(c, K); return twh::fail(c, TW_ERR_OOM, "chain blocks"); }
    TW_CUDA(c, launch_chain_blocks_f(c->Lp32, c->inv32, c->chF32, c->chB32, c->NB, s));
    TW_CUDA(c, cudaStreamSynchronize(s));
    twh::dfree(c, K32);
    c->have32 = true;
    // choose the number of refinement steps on a probe right-hand side (all
    // ones): iterate until the FP64 residual stops falling by 2x or reaches
    // 1e-13 relative; online calls then run that many steps without host sync
    std::vector<double> ones(n, 1.0);
    double *probe = (double *)twh::dalloc(c, n * sizeof(double));
    if (!probe) { twh::dfree(c, K); return twh::fail(c, TW_ERR_OOM, "probe"); }
    TW_CUDA(c, cudaMemcpy(probe, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    const int NBn = c->NB;
    st = solve32(c, probe, 0, (int)n, c->fy, s);
    if (st != TW_OK) { twh::dfree(c, probe); twh::dfree(c, K); return st; }
    TW_CUDA(c, launch_f_to_dd(c->fy, c->vy, (int)n, s));
    double prev = 1e300;
    int steps = 0;
    for (int it = 0; it < 30; ++it) {
      TW_CUDA(c, launch_residual(c->Kp64, c->vy, probe, c->vr, (int)n, NBn, s));
      TW_CUDA(c, launch_sumsq(c->vr, 1, (int)n, c->d_norm, s));
      double h = 0.0;
      TW_CUDA(c, cudaMemcpyAsync(&h, c->d_norm, sizeof(double), cudaMemcpyDeviceToHost, s));
      TW_CUDA(c, cudaStreamSynchronize(s));
      const double relr = sqrt(h / (double)n);
      if (relr <= 1e-13 || relr > 0.5 * prev) break;
      prev = relr;
      st = solve32(c, c->vr, 1, (int)n, c->fy, s);
      if (st != TW_OK) { twh::dfree(c, probe); twh::dfree(c, K); return st; }
      TW_CUDA(c, launch_axpy_dd_f(c->vy, c->fy, (int)n, s));
      steps = it + 1;
    }
    c->ir_steps = std::max(1, steps);
    c->ir_probe_resid = prev;
    twh::dfree(c, probe);
  }
  if (want64) {
    if (!c->Lp64) c->Lp64 = (double *)twh::dalloc(c, nblk * blk * sizeof(double));
    if (!c->inv64) c->inv64 = (double *)twh::dalloc(c, (size_t)c->NB * blk * sizeof(double));
    if (!c->Lp64 || !c->inv64) { twh::dfree(c, K); return twh::fail(c, TW_ERR_OOM, "factor buffers"); }
    // The factorisation runs in FP64: the panels on the FP64 pipe, the
    // rank-64 trailing updates as exact products on the tensor cores
    {
      twh::Phase pc(c, TW_PH_CHOLESKY, s);
      const size_t wsb = syrk_ws_bytes_per_atom((int)np) * 2 * cholesky_tc_width();
      uint8_t *ws = (uint8_t *)twh::dalloc(c, wsb);
      int *eg = (int *)twh::dalloc(c, (size_t)syrk_exp_rows((int)np) * sizeof(int));
      if (!ws || !eg) {
        twh::dfree(c, ws); twh::dfree(c, eg); twh::dfree(c, K);
        return twh::fail(c, TW_ERR_OOM, "Cholesky update slices");
      }
      TW_CUDA(c, launch_cholesky_d(K, np, c->NB, c->inv64, c->d_err, ws, wsb, eg, s));
      TW_CUDA(c, launch_pack_d(K, np, c->Lp64, c->NB, s));
      TW_CUDA(c, cudaStreamSynchronize(s));
      twh::dfree(c, ws);
      twh::dfree(c, eg);
    }
    TW_CUDA(c, cudaStreamSynchronize(s));
    twh::dfree(c, K);                   // the dense K is no longer needed
    K = nullptr;
    st = finish_factor64(c, s);
    if (st != TW_OK) return st;
  }
  TW_CUDA(c, cudaStreamSynchronize(s));
  twh::dfree(c, K);
  st = form_gstar(c, s);
  if (st != TW_OK) return st;
  return twh::refresh_dd_factor(c, s);
}

namespace {

// tw_infer; with q (and G^ kept) also the forecast q = F_q m of each right-hand
// side, its time FFT of m taken in the same kernel as m's inverse FFT
tw_status infer_impl(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window, const double *d,
                     double *m, double *q, tw_infer_stats *stats, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nrhs < 0 || (nrhs > 0 && (!d || !m))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  const bool mixed = prec != TW_PREC_FP64;
  if (prec < 0 || prec > 2 || !c->op[TW_MAP_F][prec])
    return twh::fail(c, TW_ERR_ARG, "requested precision was not kept at tw_create");
  // solver of K y = d: the FP64 factor, or (mixed operator path with
  // TW_SOLVE_FP32_IR selected) the FP32 factor refined with the FP64 residual
  const bool use32 = mixed && c->have32 && (c->solver == TW_SOLVE_FP32_IR || !c->have64);
  if (use32 ? !c->have32 : !c->have64)
    return twh::fail(c, TW_ERR_STATE, "tw_factor_K must come before tw_infer");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int Nd = c->Nd, Nt = c->Nt, Nm = c->Nm, Nf = c->Nf;
  const void *A = c->op[TW_MAP_F][prec];
  if (stats) { stats->ir_iters = 0; stats->resid_rel = 0.0; }
  // several right-hand sides with a reserved batch: batched solves and products
  if (nrhs > 1 && c->lane.bmax > 0 && c->inv_dd && c->have64 && !use32) {
    tw_status st = twb::infer_host_windows(c, prec, nrhs, nt_window, d, m, s);
    if (st != TW_OK || !stats) return st;
    // residual of the last right-hand side (its solution is the batch's last column)
    const int last = (nrhs - 1) % c->lane.bmax;
    const int w = nt_window ? nt_window[nrhs - 1] : Nt;
    const int nrows = Nd * w;
    const int NBw = (nrows + NB_ - 1) / NB_;
    const double *dr = d + (size_t)(nrhs - 1) * Nt * Nd;
    // the batched solves leave y as float pairs (FP64 path: in the lane's 8-byte solve buffer)
    const dd *ylast = (mixed ? c->lane.byd : reinterpret_cast<const dd *>(c->lane.by)) + (size_t)last * c->n_pad;
    TW_CUDA(c, cudaMemcpyAsync(c->vy, ylast, (size_t)nrows * sizeof(dd), cudaMemcpyDeviceToDevice, s));
    if (!c->Kp64) {   // factor loaded from a checkpoint: K itself is not held
      stats->resid_rel = -1.0;
      return TW_OK;
    }
    TW_CUDA(c, launch_residual(c->Kp64, c->vy, dr, c->vr, nrows, NBw, s));
    TW_CUDA(c, launch_sumsq(c->vr, 1, nrows, c->d_norm, s));
    TW_CUDA(c, launch_sumsq(dr, 0, nrows, c->d_norm + 1, s));
    double h[2];
    TW_CUDA(c, cudaMemcpyAsync(h, c->d_norm, sizeof(h), cudaMemcpyDeviceToHost, s));
    TW_CUDA(c, cudaStreamSynchronize(s));
    stats->resid_rel = h[1] > 0 ? sqrt(h[0] / h[1]) : 0.0;
    return TW_OK;
  }
  for (int r = 0; r < nrhs; ++r) {
    const int w = nt_window ? nt_window[r] : Nt;
    if (w < 1 || w > Nt) return twh::fail(c, TW_ERR_ARG, "window must be in [1, Nt]");
    const int nrows = Nd * w;
    const int NBw = (nrows + NB_ - 1) / NB_;
    const double *dr = d + (size_t)r * Nt * Nd;
    double *mr = m + (size_t)r * Nt * Nm;
    // 1) y = K'^{-1} d'  (leading nrows of K's factor: windows nest)
    const void *ysrc = c->yd;   // y as double (FP64 solve) or dd (refined FP32 solve)
    int ykind = 0;
    if (!use32) {
      tw_status st = solve64(c, dr, 0, nrows, c->yd, s);
      if (st != TW_OK) return st;
    } else {
      ysrc = c->vy;
      ykind = 1;
      // FP32 solve, then refinement with the FP64 residual r = d - K x
      tw_status st = solve32(c, dr, 0, nrows, c->fy, s);
      if (st != TW_OK) return st;
      TW_CUDA(c, launch_f_to_dd(c->fy, c->vy, nrows, s));
      for (int it = 0; it < c->ir_steps; ++it) {
        { twh::Phase p(c, TW_PH_RESIDUAL, s);
          TW_CUDA(c, launch_residual(c->Kp64, c->vy, dr, c->vr, nrows, NBw, s)); }
        st = solve32(c, c->vr, 1, nrows, c->fy, s);
        if (st != TW_OK) return st;
        TW_CUDA(c, launch_axpy_dd_f(c->vy, c->fy, nrows, s));
      }
      if (stats) stats->ir_iters = c->ir_steps;
    }
    if (stats && r == nrhs - 1) {
      // relative residual of the last right-hand side: |d - K y| / |d|
      if (c->Kp64 != nullptr) {
        if (!use32) TW_CUDA(c, launch_double_to_dd_vec(c->yd, c->vy, nrows, s));
        TW_CUDA(c, launch_residual(c->Kp64, c->vy, dr, c->vr, nrows, NBw, s));
        TW_CUDA(c, launch_sumsq(c->vr, 1, nrows, c->d_norm, s));
        TW_CUDA(c, launch_sumsq(dr, 0, nrows, c->d_norm + 1, s));
        double h[2];
        TW_CUDA(c, cudaMemcpyAsync(h, c->d_norm, sizeof(h), cudaMemcpyDeviceToHost, s));
        TW_CUDA(c, cudaStreamSynchronize(s));
        stats->resid_rel = h[1] > 0 ? sqrt(h[0] / h[1]) : 0.0;
      } else {
        stats->resid_rel = -1.0;
      }
    }
    // 2) x = F'^T y over the window (y rows >= w are zero), 3) m = Gamma_pr x;
    // with G^ kept, m = G'^* y in one adjoint (no prior filter)
    const void *AG = c->opG[prec];
    const int Nq = c->Nq;
    double *qr = q ? q + (size_t)r * Nt * Nq : nullptr;
    if (AG && !mixed) {
      { twh::Phase p(c, TW_PH_RFFT_DATA, s);
        TW_CUDA(c, launch_rfft_time_dd(ysrc, ykind, Nd, w, c->wr, Nd, Nd, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
        TW_CUDA(c, launch_gemv_adj_dd(AG, FMT_DD, c->wr, c->wf, Nf, Nd, Nm, s)); }
      if (qr) {
        // m, and m^ (in place of x^) for the forecast
        { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
          TW_CUDA(c, launch_irfft_rfft_time_dd(c->wf, Nm, mr, 0, Nm, c->wf, Nm, Nm, w, c->plT, c->twT,
                                               c->twL, s)); }
        { twh::Phase p(c, TW_PH_GEMV_FWD, s);
          TW_CUDA(c, launch_gemv_fwd_dd(c->op[TW_MAP_FQ][0], FMT_DD, c->wf, c->part, c->wr, Nf, Nq, Nm, s)); }
        { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
          TW_CUDA(c, launch_irfft_time_dd(c->wr, Nq, qr, 0, Nq, Nq, Nt, c->plT, c->twT, c->twL, s)); }
      } else {
        twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
        TW_CUDA(c, launch_irfft_time_dd(c->wf, Nm, mr, 0, Nm, Nm, w, c->plT, c->twT, c->twL, s));
      }
    } else if (AG) {
      // reduced-precision operator, data side in double-float (see the else branch)
      cf *wf = (cf *)c->wf;
      { twh::Phase p(c, TW_PH_RFFT_DATA, s);
        TW_CUDA(c, launch_rfft_time_dd(ysrc, ykind, Nd, w, c->wr, Nd, Nd, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
        TW_CUDA(c, launch_gemv_adj_cx(AG, (int)prec, c->wr, wf, Nf, Nd, Nm, s)); }
      if (qr) {
        cf *wr = (cf *)c->wr, *part = (cf *)c->part;
        { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
          TW_CUDA(c, launch_irfft_rfft_time_f(wf, Nm, mr, 0, Nm, wf, Nm, Nm, w, c->plT, c->twTf, c->twLf, s)); }
        { twh::Phase p(c, TW_PH_GEMV_FWD, s);
          TW_CUDA(c, launch_gemv_fwd_f(c->op[TW_MAP_FQ][prec], (int)prec, wf, part, wr, Nf, Nq, Nm, s)); }
        { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
          TW_CUDA(c, launch_irfft_time_f(wr, Nq, qr, 0, Nq, Nq, Nt, c->plT, c->twTf, c->twLf, s)); }
      } else {
        twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
        TW_CUDA(c, launch_irfft_time_f(wf, Nm, mr, 0, Nm, Nm, w, c->plT, c->twTf, c->twLf, s));
      }
    } else if (!mixed) {
      { twh::Phase p(c, TW_PH_RFFT_DATA, s);
        TW_CUDA(c, launch_rfft_time_dd(ysrc, ykind, Nd, w, c->wr, Nd, Nd, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
        TW_CUDA(c, launch_gemv_adj_dd(A, FMT_DD, c->wr, c->wf, Nf, Nd, Nm, s)); }
      { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
        TW_CUDA(c, launch_irfft_time_dd(c->wf, Nm, c->wt, 1, Nm, Nm, w, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_PRIOR, s);
        TW_CUDA(c, launch_prior_dd(c->wt, 1, mr, 0, w, c->Nx, c->Ny, c->ws, c->lam1, c->plX, c->plY,
                                   c->twX, c->twY, s)); }
    } else {
      // reduced-precision operator: y's spectrum stays double-float (y is large
      // against m, and F^T y cancels), the product forms exact products and a
      // double-float running sum; x^ onwards (inverse FFT, prior) runs in FP32
      cf *wf = (cf *)c->wf;
      float *wt = (float *)c->wt;
      { twh::Phase p(c, TW_PH_RFFT_DATA, s);
        TW_CUDA(c, launch_rfft_time_dd(ysrc, ykind, Nd, w, c->wr, Nd, Nd, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
        TW_CUDA(c, launch_gemv_adj_cx(A, (int)prec, c->wr, wf, Nf, Nd, Nm, s)); }
      { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
        TW_CUDA(c, launch_irfft_time_f(wf, Nm, wt, 2, Nm, Nm, w, c->plT, c->twTf, c->twLf, s)); }
      { twh::Phase p(c, TW_PH_PRIOR, s);
        TW_CUDA(c, launch_prior_f(wt, 2, mr, 0, w, c->Nx, c->Ny, (cf *)c->ws, c->lam1f, c->plX,
                                  c->plY, c->twXf, c->twYf, s)); }
    }
    if (w < Nt && !(qr && AG))   // the fused kernel writes the zero rows itself
      TW_CUDA(c, cudaMemsetAsync(mr + (size_t)w * Nm, 0, (size_t)(Nt - w) * Nm * sizeof(double), s));
    if (qr && !AG) {
      tw_status st = tw_p2o_apply(c, TW_MAP_FQ, prec, 1, mr, qr, stream);
      if (st != TW_OK) return st;
    }
  }
  return TW_OK;
}

}  // namespace

tw_status tw_infer(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window, const double *d,
                   double *m, tw_infer_stats *stats, void *stream) {
  return infer_impl(c, prec, nrhs, nt_window, d, m, nullptr, stats, stream);
}

tw_status tw_infer_forecast(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window, const double *d,
                            double *m, double *q, tw_infer_stats *stats, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nrhs < 0 || (nrhs > 0 && !q)) return twh::fail(c, TW_ERR_ARG, "bad forecast output");
  if (prec < 0 || prec > 2 || !c->op[TW_MAP_FQ][prec])
    return twh::fail(c, TW_ERR_ARG, "requested precision was not kept at tw_create");
  for (char l : c->loaded[TW_MAP_FQ])
    if (!l) return twh::fail(c, TW_ERR_STATE, "block column not fully loaded");
  // several right-hand sides with a reserved batch: the batched paths, one after the other
  if (nrhs > 1 && c->lane.bmax > 0) {
    tw_status st = infer_impl(c, prec, nrhs, nt_window, d, m, nullptr, stats, stream);
    return st != TW_OK ? st : tw_forecast(c, prec, nrhs, m, q, stream);
  }
  return infer_impl(c, prec, nrhs, nt_window, d, m, q, stats, stream);
}

tw_status tw_solve_K(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window, const double *d,
                     double *y, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nrhs < 0 || (nrhs > 0 && (!d || !y))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  const bool use32 = prec != TW_PREC_FP64 && c->have32 && (c->solver == TW_SOLVE_FP32_IR || !c->have64);
  if (use32 ? !c->have32 : !c->have64)
    return twh::fail(c, TW_ERR_STATE, "tw_factor_K must come before tw_solve_K");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int Nd = c->Nd, Nt = c->Nt;
  for (int r = 0; r < nrhs; ++r) {
    const int w = nt_window ? nt_window[r] : Nt;
    if (w < 1 || w > Nt) return twh::fail(c, TW_ERR_ARG, "window must be in [1, Nt]");
    const int nrows = Nd * w, NBw = (nrows + NB_ - 1) / NB_;
    const double *dr = d + (size_t)r * Nt * Nd;
    double *yr = y + (size_t)r * Nt * Nd;
    tw_status st;
    if (!use32) {
      st = solve64(c, dr, 0, nrows, c->yd, s);
      if (st != TW_OK) return st;
      TW_CUDA(c, cudaMemcpyAsync(yr, c->yd, (size_t)nrows * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      st = solve32(c, dr, 0, nrows, c->fy, s);
      if (st != TW_OK) return st;
      TW_CUDA(c, launch_f_to_dd(c->fy, c->vy, nrows, s));
      for (int it = 0; it < c->ir_steps; ++it) {
        TW_CUDA(c, launch_residual(c->Kp64, c->vy, dr, c->vr, nrows, NBw, s));
        st = solve32(c, c->vr, 1, nrows, c->fy, s);
        if (st != TW_OK) return st;
        TW_CUDA(c, launch_axpy_dd_f(c->vy, c->fy, nrows, s));
      }
      TW_CUDA(c, launch_dd_to_double(c->vy, yr, nrows, s));
    }
    if (w < Nt) TW_CUDA(c, cudaMemsetAsync(yr + nrows, 0, (size_t)(Nt - w) * Nd * sizeof(double), s));
  }
  return TW_OK;
}

tw_status tw_apply_K(tw_ctx *c, int nrhs, const int *nt_window, const double *x, double *out,
                     void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nrhs < 0 || (nrhs > 0 && (!x || !out))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  if (!c->Kp64) return twh::fail(c, TW_ERR_STATE, "tw_factor_K must come before tw_apply_K");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int Nd = c->Nd, Nt = c->Nt;
  for (int r = 0; r < nrhs; ++r) {
    const int w = nt_window ? nt_window[r] : Nt;
    if (w < 1 || w > Nt) return twh::fail(c, TW_ERR_ARG, "window must be in [1, Nt]");
    const int nrows = Nd * w, NBw = (nrows + NB_ - 1) / NB_;
    TW_CUDA(c, launch_double_to_dd_vec(x + (size_t)r * Nt * Nd, c->vz, nrows, s));
    TW_CUDA(c, launch_residual(c->Kp64, c->vz, nullptr, c->vr, nrows, NBw, s));
    double *o = out + (size_t)r * Nt * Nd;
    TW_CUDA(c, launch_dd_to_double(c->vr, o, nrows, s));
    if (w < Nt) TW_CUDA(c, cudaMemsetAsync(o + nrows, 0, (size_t)(Nt - w) * Nd * sizeof(double), s));
  }
  return TW_OK;
}

tw_status tw_sample_posterior(tw_ctx *c, int ns, const int *nt_window, const double *d,
                              const double *z_m, const double *z_n, double sigma, double *samples,
                              void *stream) {
  if (!c) return TW_ERR_ARG;
  if (ns < 0 || (ns > 0 && (!d || !z_m || !z_n || !samples)))
    return twh::fail(c, TW_ERR_ARG, "bad sample arguments");
  if (!(sigma >= 0.0)) return twh::fail(c, TW_ERR_ARG, "sigma must be >= 0");
  if (!c->have64 || !c->op[TW_MAP_F][FMT_DD])
    return twh::fail(c, TW_ERR_STATE, "tw_sample_posterior needs the FP64 factor and operator");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  if (ns > 1 && c->lane.bmax > 0)
    return twb::sample_host_windows(c, ns, nt_window, d, z_m, z_n, sigma, samples, s);
  const int Nd = c->Nd, Nt = c->Nt, Nm = c->Nm, Nf = c->Nf;
  const void *A = c->op[TW_MAP_F][FMT_DD];
  for (int k = 0; k < ns; ++k) {
    const int w = nt_window ? nt_window[k] : Nt;
    if (w < 1 || w > Nt) return twh::fail(c, TW_ERR_ARG, "window must be in [1, Nt]");
    const int nrows = Nd * w;
    const size_t off_m = (size_t)k * Nt * Nm, off_d = (size_t)k * Nt * Nd;
    double *sk = samples + off_m;
    // m_pr = Gamma_pr^{1/2} z_m  (written to the output, which accumulates the sample)
    { twh::Phase p(c, TW_PH_PRIOR, s);
      TW_CUDA(c, launch_prior_dd(z_m + off_m, 0, sk, 0, Nt, c->Nx, c->Ny, c->ws, c->lamh, c->plX,
                                 c->plY, c->twX, c->twY, s)); }
    // a = F' m_pr (leading w blocks: they depend on m_pr[0..w-1] only)
    { twh::Phase p(c, TW_PH_RFFT_PARAM, s);
      TW_CUDA(c, launch_rfft_time_dd(sk, 0, Nm, w, c->wf, Nm, Nm, c->plT, c->twT, c->twL, s)); }
    { twh::Phase p(c, TW_PH_GEMV_FWD, s);
      TW_CUDA(c, launch_gemv_fwd_dd(A, FMT_DD, c->wf, c->part, c->wr, Nf, Nd, Nm, s)); }
    { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
      TW_CUDA(c, launch_irfft_time_dd(c->wr, Nd, c->ad, 0, Nd, Nd, w, c->plT, c->twT, c->twL, s)); }
    // r = d' - F' m_pr - sigma z_n,  y = K'^{-1} r
    TW_CUDA(c, launch_sample_rhs(d + off_d, c->ad, z_n + off_d, sigma, c->rd, nrows, s));
    tw_status st = solve64(c, c->rd, 0, nrows, c->yd, s);
    if (st != TW_OK) return st;
    // s = m_pr + Gamma_pr F'^T y  (rows t >= w keep the prior draw)
    { twh::Phase p(c, TW_PH_RFFT_DATA, s);
      TW_CUDA(c, launch_rfft_time_dd(c->yd, 0, Nd, w, c->wr, Nd, Nd, c->plT, c->twT, c->twL, s)); }
    { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
      TW_CUDA(c, launch_gemv_adj_dd(A, FMT_DD, c->wr, c->wf, Nf, Nd, Nm, s)); }
    { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
      TW_CUDA(c, launch_irfft_time_dd(c->wf, Nm, c->wt, 1, Nm, Nm, w, c->plT, c->twT, c->twL, s)); }
    { twh::Phase p(c, TW_PH_PRIOR, s);
      TW_CUDA(c, launch_prior_dd(c->wt, 1, c->wt, 1, w, c->Nx, c->Ny, c->ws, c->lam1, c->plX,
                                 c->plY, c->twX, c->twY, s)); }
    TW_CUDA(c, launch_add_dd(sk, c->wt, (long)w * Nm, s));
  }
  return TW_OK;
}

tw_status tw_forecast(tw_ctx *c, tw_prec prec, int nrhs, const double *m, double *q, void *stream) {
  if (c && nrhs > 1 && c->lane.bmax > 0 && prec >= 0 && prec <= 2 && c->op[TW_MAP_FQ][prec] && m && q) {
    for (char l : c->loaded[TW_MAP_FQ])
      if (!l) return twh::fail(c, TW_ERR_STATE, "block column not fully loaded");
    TW_CUDA(c, cudaSetDevice(c->dev));
    return twb::forecast_full(c, prec, nrhs, m, q, (cudaStream_t)stream);
  }
  return tw_p2o_apply(c, TW_MAP_FQ, prec, nrhs, m, q, stream);
}

tw_status tw_set_refinement(tw_ctx *c, int steps) {
  if (!c) return TW_ERR_ARG;
  if (steps < 0 || steps > 50) return twh::fail(c, TW_ERR_ARG, "refinement steps must be in [0, 50]");
  c->ir_steps = steps;
  return TW_OK;
}

int tw_refinement_steps(const tw_ctx *c) { return c ? c->ir_steps : -1; }

tw_status tw_set_solver(tw_ctx *c, tw_solver solver) {
  if (!c) return TW_ERR_ARG;
  if (solver != TW_SOLVE_FACTOR64 && solver != TW_SOLVE_FP32_IR)
    return twh::fail(c, TW_ERR_ARG, "unknown solver");
  c->solver = solver;
  return TW_OK;
}

size_t tw_factor_bytes(const tw_ctx *c) {
  if (!c || !c->have64) return 0;
  return sizeof(FactorHeader) + factor_payload(c->NB);
}

tw_status tw_save_factor(tw_ctx *c, void *host, size_t bytes, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (!c->have64) return twh::fail(c, TW_ERR_STATE, "no FP64 factor to save (tw_factor_K first)");
  const size_t need = tw_factor_bytes(c);
  if (!host || bytes < need) return twh::fail(c, TW_ERR_ARG, "checkpoint buffer too small");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  FactorHeader h{};
  memcpy(h.magic, kFactorMagic, sizeof(h.magic));
  h.Nd = c->Nd; h.Nt = c->Nt; h.Nx = c->Nx; h.Ny = c->Ny; h.NB = c->NB; h.blk = NB_;
  h.nblk = (uint64_t)c->NB * (c->NB + 1) / 2;
  h.sigma2 = c->sigma2; h.nu = c->nu; h.ell = c->ell; h.var = c->var; h.Lx = c->Lx; h.Ly = c->Ly;
  h.col_hash = twh::column_fingerprint(c);
  uint8_t *dst = (uint8_t *)host;
  memcpy(dst, &h, sizeof(h));
  const size_t lp = (size_t)h.nblk * NB_ * NB_ * sizeof(double);
  TW_CUDA(c, cudaMemcpyAsync(dst + sizeof(h), c->Lp64, lp, cudaMemcpyDeviceToHost, s));
  TW_CUDA(c, cudaMemcpyAsync(dst + sizeof(h) + lp, c->inv64, (size_t)c->NB * NB_ * NB_ * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
  TW_CUDA(c, cudaStreamSynchronize(s));
  return TW_OK;
}

tw_status tw_load_factor(tw_ctx *c, const void *host, size_t bytes, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (!host || bytes < sizeof(FactorHeader)) return twh::fail(c, TW_ERR_ARG, "checkpoint too short");
  if (!c->prior_set) return twh::fail(c, TW_ERR_STATE, "tw_set_prior must come before tw_load_factor");
  FactorHeader h;
  memcpy(&h, host, sizeof(h));
  if (memcmp(h.magic, kFactorMagic, sizeof(h.magic)) != 0)
    return twh::fail(c, TW_ERR_ARG, "not a factor checkpoint");
  const int NB = (c->Nd * c->Nt + NB_ - 1) / NB_;
  if (h.Nd != c->Nd || h.Nt != c->Nt || h.Nx != c->Nx || h.Ny != c->Ny || h.blk != NB_ || h.NB != NB ||
      h.nblk != (uint64_t)NB * (NB + 1) / 2)
    return twh::fail(c, TW_ERR_ARG, "checkpoint was made for other sizes");
  if (h.nu != c->nu || h.ell != c->ell || h.var != c->var || h.Lx != c->Lx || h.Ly != c->Ly)
    return twh::fail(c, TW_ERR_ARG, "checkpoint was made with another prior or domain");
  if (!(h.sigma2 >= 0.0)) return twh::fail(c, TW_ERR_ARG, "checkpoint noise variance invalid");
  for (char l : c->loaded[TW_MAP_F])
    if (!l) return twh::fail(c, TW_ERR_STATE, "load the block column of F before the factor");
  if (h.col_hash != twh::column_fingerprint(c))
    return twh::fail(c, TW_ERR_ARG, "checkpoint was formed from another block column of F");
  if (bytes < sizeof(FactorHeader) + factor_payload(NB))
    return twh::fail(c, TW_ERR_ARG, "checkpoint truncated");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  TW_CUDA(c, cudaDeviceSynchronize());
  c->have64 = c->have32 = false;
  c->have_qoi = false;
  // K itself is not part of the checkpoint: a K held from an earlier
  // factorisation would not match the loaded factor
  twh::dfree(c, c->Kp64);
  c->Kp64 = nullptr;
  twh::dfree(c, c->G);      // G is only needed to form K
  c->G = nullptr;
  std::fill(c->g_rows.begin(), c->g_rows.end(), 0);
  c->n = c->Nd * c->Nt;
  c->NB = NB;
  c->n_pad = NB * NB_;
  c->sigma2 = h.sigma2;
  tw_status st = ensure_solve_workspace(c);
  if (st != TW_OK) return st;
  const size_t blk = (size_t)NB_ * NB_;
  const size_t lp = (size_t)h.nblk * blk * sizeof(double);
  if (!c->Lp64) c->Lp64 = (double *)twh::dalloc(c, lp);
  if (!c->inv64) c->inv64 = (double *)twh::dalloc(c, (size_t)NB * blk * sizeof(double));
  if (!c->Lp64 || !c->inv64) return twh::fail(c, TW_ERR_OOM, "factor buffers");
  const uint8_t *src = (const uint8_t *)host + sizeof(FactorHeader);
  TW_CUDA(c, cudaMemcpyAsync(c->Lp64, src, lp, cudaMemcpyHostToDevice, s));
  TW_CUDA(c, cudaMemcpyAsync(c->inv64, src + lp, (size_t)NB * blk * sizeof(double),
                             cudaMemcpyHostToDevice, s));
  st = finish_factor64(c, s);
  if (st != TW_OK) return st;
  st = form_gstar(c, s);
  if (st != TW_OK) return st;
  return twh::refresh_dd_factor(c, s);
}

}  // extern "C"
