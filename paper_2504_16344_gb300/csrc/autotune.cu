// autotune.cu -- tile choice of the batched per-frequency products by measurement.
//
// The batched products (the posterior mean's adjoint F^H Y and the
// forecast's forward product F_q X, one matrix product per frequency) have
// tile parameters whose best value depends on the shapes: the number of
// right-hand sides per tensor-core tile of the mixed adjoint (how many tiles
// re-read the operator against the MMA width), the right-hand sides per warp
// of the FP64-class adjoint, and the lanes per right-hand side of the
// forward products.  tw_reserve_batch times every legal candidate on the
// context's own operator and workspaces with CUDA events (one warm-up launch,
// then the mean of two) and keeps the fastest; the choice is cached for the
// process by shape, so later contexts of the same shape skip the
// measurement.  TW_AUTOTUNE=0 in the environment keeps the built-in rules.
// None of the parameters changes a result's dependence on its batch mates:
// each column's sums run in an order fixed by the parameters alone.
#include <stdlib.h>
#include <string.h>

#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "ctx.h"

using namespace tw;

namespace {

using Key = std::array<long, 7>;
std::mutex g_mu;
std::map<Key, tw_tiles> g_cache;

Key key_of(const tw_ctx *c, int bmax) {
  return {c->Nd, c->Nq, c->Nx, c->Ny, c->Nt, bmax, (long)c->keep};
}

// mean device time of fn over two launches after one warm-up (ms; -1 on error)
template <class F>
double time_ms(F fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1.0;
  double ms = -1.0;
  if (fn() == cudaSuccess) {
    cudaEventRecord(a, 0);
    bool ok = fn() == cudaSuccess && fn() == cudaSuccess;
    cudaEventRecord(b, 0);
    float t = 0.f;
    if (ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess)
      ms = 0.5 * t;
  }
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

void apply(tw_lane &L, const tw_tiles &t) {
  L.sl_tile = t.adj_tile;
  L.adj_rw = t.adj_rw;
  L.fwd_lpb = t.fwd_lanes;
}

tw_tiles rule_tiles(const tw_lane &L) {
  tw_tiles t{};
  t.adj_tile = sl_pick_tile(L.bmax);
  t.adj_rw = 0;
  t.fwd_lanes = L.bmax <= 16 ? 2 : 1;
  t.adj_tile_ms = t.adj_rw_ms = t.fwd_lanes_ms = -1.0;
  t.tuned = 0;
  return t;
}

}  // namespace

namespace twb {

void copy_tiles(tw_lane &dst, const tw_lane &src) {
  dst.sl_tile = src.sl_tile;
  dst.adj_rw = src.adj_rw;
  dst.fwd_lpb = src.fwd_lpb;
}

tw_status autotune_lane(tw_ctx *c, tw_lane &L) {
  tw_tiles t = rule_tiles(L);
  const char *env = getenv("TW_AUTOTUNE");
  if (env && strcmp(env, "0") == 0) {
    apply(L, t);
    c->tiles = t;
    return TW_OK;
  }
  const Key key = key_of(c, L.bmax);
  {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      apply(L, it->second);
      c->tiles = it->second;
      return TW_OK;
    }
  }
  TW_CUDA(c, cudaSetDevice(c->dev));
  TW_CUDA(c, cudaDeviceSynchronize());
  const int Nd = c->Nd, Nq = c->Nq, Nm = c->Nm, Nf = c->Nf, B = L.bmax;
  // inputs of the timed products: zeros (the work does not depend on values)
  TW_CUDA(c, cudaMemset(L.byh, 0, (size_t)B * Nf * c->Rmax * sizeof(cdd)));
  TW_CUDA(c, cudaMemset(L.bxh, 0, (size_t)B * Nf * Nm * sizeof(cdd)));
  // 1) mixed adjoint: right-hand sides per tensor-core tile
  const int fmt = c->op[TW_MAP_F][TW_PREC_C64] ? TW_PREC_C64 : (c->op[TW_MAP_F][TW_PREC_BF16X2] ? TW_PREC_BF16X2 : -1);
  if (fmt > 0 && L.bsl_ws) {
    const void *A = c->opG[fmt] ? c->opG[fmt] : c->op[TW_MAP_F][fmt];
    const int8_t *ea = c->opG[fmt] ? c->eaG[fmt] : c->ea[TW_MAP_F][fmt];
    std::vector<int> cand;
    for (int P = 8; P <= 80 && P <= (B + 7) / 8 * 8; P += 8) cand.push_back(P);
    std::vector<double> ms;
    for (int P : cand)
      ms.push_back(time_ms([&] {
        return launch_gemm_adj_sl(A, fmt, ea, (const cdd *)L.byh, (long)Nf * Nd, (cf *)L.bxh, (long)Nf * Nm, Nf,
                                  Nd, Nm, B, P, L.bsl_ws, L.bsl_ws_n, L.bsl_eb, L.bsl_eb_n, c->d_err, 0);
      }));
    const int k = tw_autotune_pick((int)ms.size(), ms.data());
    if (k >= 0) { t.adj_tile = cand[k]; t.adj_tile_ms = ms[k]; }
  }
  // 2) FP64-class adjoint: right-hand sides per warp
  if (c->op[TW_MAP_F][TW_PREC_FP64]) {
    const void *A = c->opG[0] ? c->opG[0] : c->op[TW_MAP_F][0];
    const int cand[3] = {4, 2, 1};
    double ms[3];
    for (int k = 0; k < 3; ++k)
      ms[k] = time_ms([&] {
        return launch_gemm_adj_dd(A, (const cdd *)L.byh, (long)Nf * Nd, (cdd *)L.bxh, (long)Nf * Nm, Nf, Nd, Nm,
                                  B, 0, cand[k]);
      });
    const int k = tw_autotune_pick(3, ms);
    if (k >= 0) { t.adj_rw = cand[k]; t.adj_rw_ms = ms[k]; }
  }
  // 3) forward products (the forecast's F_q X): lanes per right-hand side
  {
    const int cand[2] = {1, 2};
    double ms[2];
    const bool f64 = c->op[TW_MAP_FQ][TW_PREC_FP64] != nullptr;
    const int ffmt = f64 ? TW_PREC_FP64 : fmt;
    for (int k = 0; k < 2; ++k)
      ms[k] = ffmt < 0 ? -1.0 : time_ms([&] {
        if (f64)
          return launch_gemm_fwd_dd(c->op[TW_MAP_FQ][0], (const cdd *)L.bxh, (long)Nf * Nm, (cdd *)L.bpart,
                                    (cdd *)L.byh, (long)Nf * Nq, Nf, Nq, Nm, B, 0, cand[k]);
        return launch_gemm_fwd_f(c->op[TW_MAP_FQ][ffmt], ffmt, (const cf *)L.bxh, (long)Nf * Nm, (cf *)L.bpart,
                                 (cf *)L.byh, (long)Nf * Nq, Nf, Nq, Nm, B, 0, cand[k]);
      });
    const int k = tw_autotune_pick(2, ms);
    if (k >= 0) { t.fwd_lanes = cand[k]; t.fwd_lanes_ms = ms[k]; }
  }
  TW_CUDA(c, cudaDeviceSynchronize());
  tw_status st = tw_check(c, 0);
  if (st != TW_OK) return st;
  t.tuned = 1;
  apply(L, t);
  c->tiles = t;
  std::lock_guard<std::mutex> g(g_mu);
  g_cache[key] = t;
  return TW_OK;
}

}  // namespace twb

extern "C" {

int tw_autotune_pick(int n, const double *ms) {
  int best = -1;
  for (int k = 0; k < n; ++k)
    if (ms && ms[k] > 0.0 && (best < 0 || ms[k] < ms[best])) best = k;
  return best;
}

tw_status tw_batch_tiles(const tw_ctx *c, tw_tiles *out) {
  if (!c || !out) return TW_ERR_ARG;
  if (c->lane.bmax <= 0) return TW_ERR_STATE;
  *out = c->tiles;
  return TW_OK;
}

tw_status tw_set_batch_tiles(tw_ctx *c, const tw_tiles *t) {
  if (!c || !t) return TW_ERR_ARG;
  if (c->lane.bmax <= 0) return twh::fail(c, TW_ERR_STATE, "tw_reserve_batch must come first");
  if (t->adj_tile < 8 || t->adj_tile > 80 || t->adj_tile % 8 != 0)
    return twh::fail(c, TW_ERR_ARG, "adj_tile must be a multiple of 8 in [8, 80]");
  if (t->adj_rw != 0 && t->adj_rw != 1 && t->adj_rw != 2 && t->adj_rw != 4)
    return twh::fail(c, TW_ERR_ARG, "adj_rw must be 0, 1, 2 or 4");
  if (t->fwd_lanes != 1 && t->fwd_lanes != 2) return twh::fail(c, TW_ERR_ARG, "fwd_lanes must be 1 or 2");
  tw_tiles v = *t;
  v.adj_tile_ms = v.adj_rw_ms = v.fwd_lanes_ms = -1.0;
  v.tuned = 2;
  apply(c->lane, v);
  c->tiles = v;
  return TW_OK;
}

void tw_autotune_clear_cache(void) {
  std::lock_guard<std::mutex> g(g_mu);
  g_cache.clear();
}

}  // extern "C"
