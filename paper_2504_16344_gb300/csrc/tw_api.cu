// tw_api.cu -- context, operator set-up, Toeplitz applies and the prior.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "ctx.h"

using namespace tw;

namespace tw {
static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace tw

// splitmix64 finaliser (Steele, Lea and Flood 2014): a well-mixed 64-bit hash
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

namespace twh {

static cudaEvent_t get_event(tw_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

Phase::Phase(tw_ctx *c_, int ph_, cudaStream_t s_) : c(c_), ph(ph_), s(s_) {
  if (c && c->prof) {
    a = get_event(c);
    cudaEventRecord(a, s);
  }
}

Phase::~Phase() {
  if (a) {
    cudaEvent_t b = get_event(c);
    cudaEventRecord(b, s);
    c->prof_pending.push_back({ph, a, b});
  }
}

tw_status fail(tw_ctx *c, tw_status st, const std::string &msg) {
  if (c) c->err = msg;
  return st;
}

tw_status cuda_fail(tw_ctx *c, cudaError_t e, const char *where) {
  std::string m = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + where;
  return fail(c, e == cudaErrorMemoryAllocation ? TW_ERR_OOM : TW_ERR_CUDA, m);
}

void *dalloc(tw_ctx *c, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->allocs.push_back(p);
  c->alloc_sizes.push_back(bytes);
  c->bytes += bytes;
  return p;
}

void dfree(tw_ctx *c, void *p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) {
    const size_t i = it - c->allocs.begin();
    c->bytes -= c->alloc_sizes[i];
    c->alloc_sizes.erase(c->alloc_sizes.begin() + i);
    c->allocs.erase(it);
  }
  cudaFree(p);
}

// Factor M into radices: 4s first, then 2, 3, 5, 7, then remaining odd primes.
FftPlan make_plan(int M) {
  FftPlan p{};
  p.M = M;
  int m = M, n = 0;
  const int small[5] = {4, 2, 3, 5, 7};
  for (int r : small)
    while (m % r == 0 && n < TW_FFT_MAX_STAGES) { p.R[n++] = r; m /= r; }
  for (int q = 11; m > 1 && n < TW_FFT_MAX_STAGES; q += 2)
    while (m % q == 0 && n < TW_FFT_MAX_STAGES) { p.R[n++] = q; m /= q; }
  if (m > 1) p.R[n++] = m;  // remaining factor (only for absurd lengths)
  p.nst = n;
  // magic multipliers for the engine's divisions by p and by S = M / R
  auto mag = [](unsigned x) -> unsigned { return x <= 1 ? 0u : (unsigned)((1ull << 32) / x); };
  int prod = 1;
  for (int st = 0; st < n; ++st) {
    p.pmag[st] = mag((unsigned)prod);
    p.smag[st] = mag((unsigned)(M / p.R[st]));
    prod *= p.R[st];
  }
  return p;
}

unsigned long long column_fingerprint(const tw_ctx *c) {
  unsigned long long h = 0x5457u;
  for (size_t r = 0; r < c->col_hash.size(); ++r) h = mix64(h ^ mix64(c->col_hash[r] + r));
  return h;
}

}  // namespace twh

namespace {

const double kPi = 3.14159265358979323846;

void split_dd(double v, dd &o) {
  o.hi = (float)v;
  o.lo = (float)(v - (double)o.hi);
}

// W_M^t = exp(-2 pi i t / M) for t < n (n = M, or M+1 with denominator 2M)
tw_status upload_twiddles(tw_ctx *c, int n, double denom, cdd **out_dd, cf **out_f) {
  std::vector<cdd> h(n);
  std::vector<cf> hf(n);
  for (int t = 0; t < n; ++t) {
    const double a = -2.0 * kPi * (double)t / denom;
    const double cr = cos(a), ci = sin(a);
    split_dd(cr, h[t].re);
    split_dd(ci, h[t].im);
    hf[t].re = (float)cr;
    hf[t].im = (float)ci;
  }
  *out_dd = (cdd *)twh::dalloc(c, n * sizeof(cdd));
  *out_f = (cf *)twh::dalloc(c, n * sizeof(cf));
  if (!*out_dd || !*out_f) return twh::fail(c, TW_ERR_OOM, "twiddle allocation");
  TW_CUDA(c, cudaMemcpy(*out_dd, h.data(), n * sizeof(cdd), cudaMemcpyHostToDevice));
  TW_CUDA(c, cudaMemcpy(*out_f, hf.data(), n * sizeof(cf), cudaMemcpyHostToDevice));
  return TW_OK;
}

tw_status upload_twiddles_d(tw_ctx *c, int n, double denom, cd **out) {
  std::vector<cd> h(n);
  for (int t = 0; t < n; ++t) {
    const double a = -2.0 * kPi * (double)t / denom;
    h[t].re = cos(a);
    h[t].im = sin(a);
  }
  *out = (cd *)twh::dalloc(c, n * sizeof(cd));
  if (!*out) return twh::fail(c, TW_ERR_OOM, "twiddle allocation");
  TW_CUDA(c, cudaMemcpy(*out, h.data(), n * sizeof(cd), cudaMemcpyHostToDevice));
  return TW_OK;
}

// G rows for F's block-column rows [row0, row0+nrows): G[t*Nd + row0 + r] =
// C^{1/2} F_t[r, :], native FP64 filter, stored as float pairs.
tw_status build_G_rows(tw_ctx *c, int row0, int nrows, const double *col, cudaStream_t s) {
  const int Nt = c->Nt, Nd = c->Nd, Nm = c->Nm;
  if (!c->G) {
    c->G = (dd *)twh::dalloc(c, (size_t)Nt * Nd * Nm * sizeof(dd));
    if (!c->G) return twh::fail(c, TW_ERR_OOM, "G buffer (tw_set_prior before tw_set_block_column)");
  }
  const int cap = 2 * ((Nt + 1) / 2);    // fields the spatial workspace holds
  if (nrows <= cap) {
    const int lags = cap / nrows;
    for (int u0 = 0; u0 < Nt; u0 += lags) {
      const int nl = std::min(lags, Nt - u0);
      TW_CUDA(c, launch_prior_d(col + (size_t)u0 * nrows * Nm, 0, c->G, 1, nl * nrows, c->Nx, c->Ny,
                                (cd *)c->ws, c->lamhd, c->plX, c->plY, c->twXd, c->twYd, nrows,
                                Nd, u0 * Nd + row0, s));
    }
  } else {
    for (int u = 0; u < Nt; ++u)
      for (int r0 = 0; r0 < nrows; r0 += cap) {
        const int nr = std::min(cap, nrows - r0);
        TW_CUDA(c, launch_prior_d(col + ((size_t)u * nrows + r0) * Nm, 0, c->G, 1, nr, c->Nx,
                                  c->Ny, (cd *)c->ws, c->lamhd, c->plX, c->plY, c->twXd, c->twYd,
                                  1 << 30, 0, u * Nd + row0 + r0, s));
      }
  }
  for (int r = row0; r < row0 + nrows; ++r) c->g_rows[r] = 1;
  return TW_OK;
}

// per-row fingerprint of a block-column chunk [Nt][nrows][Nm]: the sum over
// its entries of mix64(bits ^ mix64(position in the row)), so that a
// checkpoint can tell whether it was formed from the same operator
__global__ void k_col_hash(const double *__restrict__ col, int nrows, int Nm,
                           unsigned long long *__restrict__ row_hash) {
  __shared__ unsigned long long red[256];
  const int l = blockIdx.x / nrows, r = blockIdx.x % nrows;
  const double *p = col + ((size_t)l * nrows + r) * Nm;
  unsigned long long h = 0;
  for (int k = threadIdx.x; k < Nm; k += blockDim.x)
    h += mix64((unsigned long long)__double_as_longlong(p[k]) ^ mix64((unsigned long long)l * Nm + k));
  red[threadIdx.x] = h;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(row_hash + r, red[0]);
}

size_t op_elem_bytes(int fmt) { return fmt == FMT_DD ? sizeof(cdd) : 8; }

int rows_of(const tw_ctx *c, int which) { return which == TW_MAP_F ? c->Nd : c->Nq; }

tw_status check_ready(tw_ctx *c, int which, int fmt) {
  if (!c) return TW_ERR_ARG;
  if (which != TW_MAP_F && which != TW_MAP_FQ) return twh::fail(c, TW_ERR_ARG, "bad map");
  if (fmt < 0 || fmt > 2 || !c->op[which][fmt])
    return twh::fail(c, TW_ERR_ARG, "requested precision was not kept at tw_create");
  for (char l : c->loaded[which])
    if (!l) return twh::fail(c, TW_ERR_STATE, "block column not fully loaded");
  return TW_OK;
}

}  // namespace

extern "C" {

tw_status tw_create(tw_ctx **out, int Nd, int Nq, int Nx, int Ny, int Nt, double Lx, double Ly,
                    unsigned keep, int device) {
  if (!out) return TW_ERR_ARG;
  *out = nullptr;
  if (Nd <= 0 || Nq <= 0 || Nx <= 0 || Ny <= 0 || Nt <= 0 || !(Lx > 0) || !(Ly > 0) ||
      (keep & 7u) == 0)
    return TW_ERR_ARG;
  tw_ctx *c = new tw_ctx();
  c->dev = device;
  c->Nd = Nd; c->Nq = Nq; c->Nx = Nx; c->Ny = Ny; c->Nt = Nt;
  c->Nm = Nx * Ny; c->Nf = Nt + 1; c->Rmax = std::max(Nd, Nq);
  c->Lx = Lx; c->Ly = Ly; c->keep = keep;
  c->loaded[0].assign(Nd, 0);
  c->loaded[1].assign(Nq, 0);
  c->col_hash.assign(Nd, 0ull);
  tw_status st = TW_OK;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) { st = twh::cuda_fail(c, e, "cudaSetDevice"); delete c; return st; }
  const size_t Nf = c->Nf, Nm = c->Nm;
  for (int which = 0; which < 2 && st == TW_OK; ++which)
    for (int fmt = 0; fmt < 3; ++fmt) {
      if (!(keep & (1u << fmt))) continue;
      const size_t b = Nf * (size_t)rows_of(c, which) * Nm * op_elem_bytes(fmt);
      c->op[which][fmt] = twh::dalloc(c, b);
      if (!c->op[which][fmt]) { st = twh::fail(c, TW_ERR_OOM, "operator allocation"); break; }
    }
  c->plT = twh::make_plan(Nt);
  c->plX = twh::make_plan(Nx);
  c->plY = twh::make_plan(Ny);
  if (st == TW_OK) st = upload_twiddles(c, Nt, Nt, &c->twT, &c->twTf);
  if (st == TW_OK) st = upload_twiddles(c, Nt + 1, 2.0 * Nt, &c->twL, &c->twLf);
  if (st == TW_OK) st = upload_twiddles(c, Nx, Nx, &c->twX, &c->twXf);
  if (st == TW_OK) st = upload_twiddles(c, Ny, Ny, &c->twY, &c->twYf);
  if (st == TW_OK) st = upload_twiddles_d(c, Nx, Nx, &c->twXd);
  if (st == TW_OK) st = upload_twiddles_d(c, Ny, Ny, &c->twYd);
  c->g_rows.assign(Nd, 0);
  if (st == TW_OK) {
    const int nchunk = gemv_fwd_nchunk(c->Nm);
    c->wf = (cdd *)twh::dalloc(c, Nf * Nm * sizeof(cdd));
    c->wr = (cdd *)twh::dalloc(c, Nf * c->Rmax * sizeof(cdd));
    c->part = (cdd *)twh::dalloc(c, Nf * (size_t)nchunk * c->Rmax * sizeof(cdd));
    c->wt = (dd *)twh::dalloc(c, (size_t)Nt * Nm * sizeof(dd));
    c->ws = (cdd *)twh::dalloc(c, (size_t)((Nt + 1) / 2) * Nm * sizeof(cdd));
    c->d_err = (int *)twh::dalloc(c, 4 * sizeof(int));
    if (!c->wf || !c->wr || !c->part || !c->wt || !c->ws || !c->d_err)
      st = twh::fail(c, TW_ERR_OOM, "workspace allocation");
    else if (cudaMemset(c->d_err, 0, 4 * sizeof(int)) != cudaSuccess)
      st = twh::fail(c, TW_ERR_CUDA, "memset");
  }
  if (st == TW_OK && (keep & (TW_KEEP_C64 | TW_KEEP_BF16X2))) {
    // row exponents of the FP32 storages for the batched adjoint on the tensor cores
    for (int which = 0; which < 2; ++which)
      for (int fmt = 1; fmt < 3; ++fmt)
        if (c->op[which][fmt]) {
          c->ea[which][fmt] = (int8_t *)twh::dalloc(c, Nf * Nm);
          if (!c->ea[which][fmt]) st = twh::fail(c, TW_ERR_OOM, "row exponent tables");
        }
  }
  if (st != TW_OK) {
    // keep the message for the caller: report via stderr since ctx is freed
    fprintf(stderr, "tw_create: %s\n", c->err.c_str());
    tw_destroy(c);
    return st;
  }
  *out = c;
  return TW_OK;
}

void tw_destroy(tw_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  for (auto &pe : c->prof_pending) { cudaEventDestroy(pe.a); cudaEventDestroy(pe.b); }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

const char *tw_last_error(const tw_ctx *c) { return c ? c->err.c_str() : "null context"; }

size_t tw_device_bytes(const tw_ctx *c) { return c ? c->bytes : 0; }

tw_status tw_set_block_column(tw_ctx *c, tw_map which, int row0, int nrows, const double *col,
                              void *stream) {
  if (!c) return TW_ERR_ARG;
  if (which != TW_MAP_F && which != TW_MAP_FQ) return twh::fail(c, TW_ERR_ARG, "bad map");
  const int R = rows_of(c, which);
  if (row0 < 0 || nrows <= 0 || row0 + nrows > R || !col)
    return twh::fail(c, TW_ERR_ARG, "row range outside the map or null column");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const long N = (long)nrows * c->Nm;                 // series in this chunk
  const long out_ld = (long)R * c->Nm;                // frequency row stride of F^
  cdd *dst = (cdd *)c->op[which][FMT_DD];
  cdd *tmp = nullptr;
  long dst_ld = out_ld;
  if (dst) {
    dst += (long)row0 * c->Nm;
  } else {
    tmp = (cdd *)twh::dalloc(c, (size_t)c->Nf * N * sizeof(cdd));
    if (!tmp) return twh::fail(c, TW_ERR_OOM, "temporary for block column");
    dst = tmp;
    dst_ld = N;
  }
  TW_CUDA(c, launch_rfft_time_dd(col, 0, N, c->Nt, dst, dst_ld, (int)N, c->plT, c->twT, c->twL, s));
  for (int fmt = 1; fmt < 3; ++fmt) {
    if (!c->op[which][fmt]) continue;
    uint8_t *d8 = (uint8_t *)c->op[which][fmt] + (size_t)row0 * c->Nm * 8;
    TW_CUDA(c, launch_convert_op(dst, dst_ld, d8, fmt, out_ld, N, c->Nf, s));
  }
  if (tmp) {
    TW_CUDA(c, cudaStreamSynchronize(s));
    twh::dfree(c, tmp);
  }
  for (int r = row0; r < row0 + nrows; ++r) c->loaded[which][r] = 1;
  if (which == TW_MAP_F) {
    // fingerprints of these rows of F (checked by tw_load_factor)
    unsigned long long *dh = (unsigned long long *)twh::dalloc(c, (size_t)nrows * sizeof(unsigned long long));
    if (!dh) return twh::fail(c, TW_ERR_OOM, "block-column fingerprint");
    TW_CUDA(c, cudaMemsetAsync(dh, 0, (size_t)nrows * sizeof(unsigned long long), s));
    k_col_hash<<<(unsigned)c->Nt * nrows, 256, 0, s>>>(col, nrows, c->Nm, dh);
    count_launches(1);
    TW_CUDA(c, cudaGetLastError());
    TW_CUDA(c, cudaMemcpyAsync(c->col_hash.data() + row0, dh, (size_t)nrows * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
    TW_CUDA(c, cudaStreamSynchronize(s));
    twh::dfree(c, dh);
  }
  // every row present: the row exponents of the FP32 storages (one pass)
  bool all = true;
  for (char l : c->loaded[which]) all = all && l;
  for (int fmt = 1; fmt < 3 && all; ++fmt)
    if (c->ea[which][fmt])
      TW_CUDA(c, launch_row_exp(c->op[which][fmt], fmt, c->ea[which][fmt], c->Nf, R, c->Nm, s));
  // with the prior known, keep G = Phi C^{1/2} of these rows for tw_factor_K,
  // computed in FP64 from the caller's FP64 column
  if (which == TW_MAP_F && c->prior_set) {
    tw_status st = build_G_rows(c, row0, nrows, col, s);
    if (st != TW_OK) return st;
  }
  return TW_OK;
}

tw_status tw_set_prior(tw_ctx *c, double nu, double ell, double var) {
  if (!c) return TW_ERR_ARG;
  if (!(nu > 0) || !(ell > 0) || !(var > 0)) return twh::fail(c, TW_ERR_ARG, "prior parameters must be positive");
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int Nx = c->Nx, Ny = c->Ny;
  const size_t N = (size_t)Nx * Ny;
  const double kappa = sqrt(2.0 * nu) / ell;
  std::vector<double> s(N);
  double ssum = 0.0;
  for (int p = 0; p < Nx; ++p) {
    const int pf = (p <= Nx / 2) ? p : p - Nx;          // signed frequency
    const double kx = 2.0 * kPi * pf / c->Lx;
    for (int q = 0; q < Ny; ++q) {
      const int qf = (q <= Ny / 2) ? q : q - Ny;
      const double ky = 2.0 * kPi * qf / c->Ly;
      const double v = pow(kappa * kappa + kx * kx + ky * ky, -(nu + 1.0));
      s[(size_t)p * Ny + q] = v;
      ssum += v;
    }
  }
  std::vector<dd> l1(N), lh(N);
  std::vector<float> l1f(N), lhf(N);
  std::vector<double> lhd(N), l1d(N);
  for (size_t i = 0; i < N; ++i) {
    const double lam = var * (double)N * s[i] / ssum;   // eigenvalue of C
    const double a = lam / (double)N, b = sqrt(lam) / (double)N;   // 1/N of the inverse DFT folded in
    split_dd(a, l1[i]);
    split_dd(b, lh[i]);
    l1f[i] = (float)a;
    lhf[i] = (float)b;
    lhd[i] = b;
    l1d[i] = a;
  }
  if (!c->lam1) {
    c->lam1 = (dd *)twh::dalloc(c, N * sizeof(dd));
    c->lamh = (dd *)twh::dalloc(c, N * sizeof(dd));
    c->lam1f = (float *)twh::dalloc(c, N * sizeof(float));
    c->lamhf = (float *)twh::dalloc(c, N * sizeof(float));
    c->lamhd = (double *)twh::dalloc(c, N * sizeof(double));
    c->lam1d = (double *)twh::dalloc(c, N * sizeof(double));
    if (!c->lam1 || !c->lamh || !c->lam1f || !c->lamhf || !c->lamhd || !c->lam1d)
      return twh::fail(c, TW_ERR_OOM, "prior tables");
  }
  TW_CUDA(c, cudaMemcpy(c->lamhd, lhd.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  TW_CUDA(c, cudaMemcpy(c->lam1d, l1d.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  // a new prior invalidates any G built with the old one
  std::fill(c->g_rows.begin(), c->g_rows.end(), 0);
  TW_CUDA(c, cudaMemcpy(c->lam1, l1.data(), N * sizeof(dd), cudaMemcpyHostToDevice));
  TW_CUDA(c, cudaMemcpy(c->lamh, lh.data(), N * sizeof(dd), cudaMemcpyHostToDevice));
  TW_CUDA(c, cudaMemcpy(c->lam1f, l1f.data(), N * sizeof(float), cudaMemcpyHostToDevice));
  TW_CUDA(c, cudaMemcpy(c->lamhf, lhf.data(), N * sizeof(float), cudaMemcpyHostToDevice));
  c->nu = nu; c->ell = ell; c->var = var;
  c->prior_set = true;
  return TW_OK;
}

tw_status tw_p2o_apply(tw_ctx *c, tw_map which, tw_prec prec, int nrhs, const double *x,
                       double *out, void *stream) {
  tw_status st = check_ready(c, which, (int)prec);
  if (st != TW_OK) return st;
  if (nrhs < 0 || (nrhs > 0 && (!x || !out))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int R = rows_of(c, which), Nt = c->Nt, Nf = c->Nf, Nm = c->Nm;
  const void *A = c->op[which][prec];
  for (int r = 0; r < nrhs; ++r) {
    const double *xr = x + (size_t)r * Nt * Nm;
    double *outr = out + (size_t)r * Nt * R;
    if (prec == TW_PREC_FP64) {
      { twh::Phase p(c, TW_PH_RFFT_PARAM, s);
        TW_CUDA(c, launch_rfft_time_dd(xr, 0, Nm, Nt, c->wf, Nm, Nm, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_GEMV_FWD, s);
        TW_CUDA(c, launch_gemv_fwd_dd(A, FMT_DD, c->wf, c->part, c->wr, Nf, R, Nm, s)); }
      { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
        TW_CUDA(c, launch_irfft_time_dd(c->wr, R, outr, 0, R, R, Nt, c->plT, c->twT, c->twL, s)); }
    } else {
      cf *wf = (cf *)c->wf, *wr = (cf *)c->wr, *part = (cf *)c->part;
      { twh::Phase p(c, TW_PH_RFFT_PARAM, s);
        TW_CUDA(c, launch_rfft_time_f(xr, 0, Nm, Nt, wf, Nm, Nm, c->plT, c->twTf, c->twLf, s)); }
      { twh::Phase p(c, TW_PH_GEMV_FWD, s);
        TW_CUDA(c, launch_gemv_fwd_f(A, (int)prec, wf, part, wr, Nf, R, Nm, s)); }
      { twh::Phase p(c, TW_PH_IRFFT_DATA, s);
        TW_CUDA(c, launch_irfft_time_f(wr, R, outr, 0, R, R, Nt, c->plT, c->twTf, c->twLf, s)); }
    }
  }
  return TW_OK;
}

tw_status tw_p2o_adjoint(tw_ctx *c, tw_map which, tw_prec prec, int nrhs, const double *y,
                         double *x, void *stream) {
  tw_status st = check_ready(c, which, (int)prec);
  if (st != TW_OK) return st;
  if (nrhs < 0 || (nrhs > 0 && (!x || !y))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int R = rows_of(c, which), Nt = c->Nt, Nf = c->Nf, Nm = c->Nm;
  const void *A = c->op[which][prec];
  if (prec != TW_PREC_FP64 && nrhs > 1 && c->lane.bmax > 0) {
    // several right-hand sides with a reserved batch: the per-frequency
    // products as one matrix product on the tensor cores (exact slices)
    for (int r0 = 0; r0 < nrhs; r0 += c->lane.bmax) {
      const int nb = std::min(c->lane.bmax, nrhs - r0);
      const BatchArg ba_y{nb, (long)Nt * R, (long)Nf * R, 0, nullptr};
      const BatchArg ba_x{nb, (long)Nf * Nm, (long)Nt * Nm, 0, nullptr};
      { twh::Phase p(c, TW_PH_RFFT_DATA, s);
        TW_CUDA(c, launch_rfft_time_dd(y + (size_t)r0 * Nt * R, 0, R, Nt, (cdd *)c->lane.byh, R, R, c->plT,
                                       c->twT, c->twL, s, ba_y)); }
      { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
        TW_CUDA(c, launch_gemm_adj_sl(A, (int)prec, c->ea[which][prec], (const cdd *)c->lane.byh, (long)Nf * R,
                                      (cf *)c->lane.bxh, (long)Nf * Nm, Nf, R, Nm, nb, c->lane.sl_tile, c->lane.bsl_ws,
                                      c->lane.bsl_ws_n, c->lane.bsl_eb, c->lane.bsl_eb_n, c->d_err, s)); }
      { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
        TW_CUDA(c, launch_irfft_time_f((const cf *)c->lane.bxh, Nm, x + (size_t)r0 * Nt * Nm, 0, Nm, Nm, Nt,
                                       c->plT, c->twTf, c->twLf, s, ba_x)); }
    }
    return TW_OK;
  }
  for (int r = 0; r < nrhs; ++r) {
    const double *yr = y + (size_t)r * Nt * R;
    double *xr = x + (size_t)r * Nt * Nm;
    if (prec == TW_PREC_FP64) {
      { twh::Phase p(c, TW_PH_RFFT_DATA, s);
        TW_CUDA(c, launch_rfft_time_dd(yr, 0, R, Nt, c->wr, R, R, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
        TW_CUDA(c, launch_gemv_adj_dd(A, FMT_DD, c->wr, c->wf, Nf, R, Nm, s)); }
      { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
        TW_CUDA(c, launch_irfft_time_dd(c->wf, Nm, xr, 0, Nm, Nm, Nt, c->plT, c->twT, c->twL, s)); }
    } else {
      // FP32 operator; the data-side spectrum in double-float, exact products
      // and a double-float running sum (as the posterior mean's adjoint)
      cf *wf = (cf *)c->wf;
      { twh::Phase p(c, TW_PH_RFFT_DATA, s);
        TW_CUDA(c, launch_rfft_time_dd(yr, 0, R, Nt, c->wr, R, R, c->plT, c->twT, c->twL, s)); }
      { twh::Phase p(c, TW_PH_GEMV_ADJ, s);
        TW_CUDA(c, launch_gemv_adj_cx(A, (int)prec, c->wr, wf, Nf, R, Nm, s)); }
      { twh::Phase p(c, TW_PH_IRFFT_PARAM, s);
        TW_CUDA(c, launch_irfft_time_f(wf, Nm, xr, 0, Nm, Nm, Nt, c->plT, c->twTf, c->twLf, s)); }
    }
  }
  return TW_OK;
}

tw_status tw_prior_apply(tw_ctx *c, double power, int nrhs, const double *x, double *y,
                         void *stream) {
  if (!c) return TW_ERR_ARG;
  if (!c->prior_set) return twh::fail(c, TW_ERR_STATE, "prior not set");
  if (!(power == 1.0 || power == 0.5)) return twh::fail(c, TW_ERR_ARG, "power must be 1 or 0.5");
  if (nrhs < 0 || (nrhs > 0 && (!x || !y))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const dd *lam = power == 1.0 ? c->lam1 : c->lamh;
  for (int r = 0; r < nrhs; ++r) {
    const size_t off = (size_t)r * c->Nt * c->Nm;
    twh::Phase p(c, TW_PH_PRIOR, s);
    TW_CUDA(c, launch_prior_dd(x + off, 0, y + off, 0, c->Nt, c->Nx, c->Ny, c->ws, lam, c->plX,
                               c->plY, c->twX, c->twY, s));
  }
  return TW_OK;
}

tw_status tw_profile_enable(tw_ctx *c, int on) {
  if (!c) return TW_ERR_ARG;
  c->prof = on != 0;
  return TW_OK;
}

tw_status tw_profile_read(tw_ctx *c, double *ms, long long *calls, int reset) {
  if (!c) return TW_ERR_ARG;
  TW_CUDA(c, cudaSetDevice(c->dev));
  for (auto &pe : c->prof_pending) {
    TW_CUDA(c, cudaEventSynchronize(pe.b));
    float t = 0.f;
    TW_CUDA(c, cudaEventElapsedTime(&t, pe.a, pe.b));
    c->prof_ms[pe.ph] += t;
    c->prof_calls[pe.ph] += 1;
    c->ev_pool.push_back(pe.a);
    c->ev_pool.push_back(pe.b);
  }
  c->prof_pending.clear();
  for (int i = 0; i < TW_PH_COUNT; ++i) {
    if (ms) ms[i] = c->prof_ms[i];
    if (calls) calls[i] = c->prof_calls[i];
    if (reset) { c->prof_ms[i] = 0.0; c->prof_calls[i] = 0; }
  }
  return TW_OK;
}

long long tw_kernel_launches(void) { return tw::launches_total(); }

tw_status tw_check(tw_ctx *c, void *stream) {
  if (!c) return TW_ERR_ARG;
  TW_CUDA(c, cudaSetDevice(c->dev));
  TW_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
  int h[4] = {0, 0, 0, 0};
  TW_CUDA(c, cudaMemcpy(h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[0] == 0) return TW_OK;
  TW_CUDA(c, cudaMemset(c->d_err, 0, sizeof(h)));
  char buf[160];
  if (h[0] == TW_ERR_NOT_SPD) {
    snprintf(buf, sizeof buf, "Cholesky: non-positive pivot at row %d", h[1]);
    return twh::fail(c, TW_ERR_NOT_SPD, buf);
  }
  if (h[0] == TW_ERR_TIMEOUT) {
    if (c->abort_flag) TW_CUDA(c, cudaMemset(c->abort_flag, 0, sizeof(int)));
    snprintf(buf, sizeof buf, "a bounded device wait ran out (site %d)", h[1]);
    return twh::fail(c, TW_ERR_TIMEOUT, buf);
  }
  snprintf(buf, sizeof buf, "device error code %d info %d", h[0], h[1]);
  return twh::fail(c, (tw_status)h[0], buf);
}

}  // extern "C"
