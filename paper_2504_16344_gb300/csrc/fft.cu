// fft.cu -- time-axis real FFTs and the Matern spectral filter.
//
// Time axis (Sec. "FFT-based Hessian matvecs", circulant embedding): a real
// series x_0..x_{M-1} (M = Nt) zero-padded to L = 2M is transformed with one
// complex FFT of length M on z_j = x_{2j} + i x_{2j+1} followed by the usual
// even/odd split X_k = E_k + W_L^k O_k, k = 0..M (M+1 = Nt+1 frequencies).
// Series are the contiguous axis of the time-major arrays ([time][series]),
// so a CTA reads B adjacent series row by row with coalesced loads and never
// transposes anything in HBM.
//
// Prior (Sec. "State of the art": block diagonal in time, each block a
// Matern covariance): C x = IDFT2(lambda * DFT2(x)) per time step.  Two
// time steps are packed into one complex field (C is real), and the 2D
// transform runs as rows (contiguous), columns (strided, with the lambda
// scaling and the inverse column transform fused), inverse rows.
#include <algorithm>

#include "kernels.h"

namespace tw {

namespace {

// real input loaders by kind (0 double, 1 dd, 2 float)
template <class P>
__device__ __forceinline__ typename P::re ld_in(const void *base, int kind, long off);
template <>
__device__ __forceinline__ dd ld_in<PolDD>(const void *base, int kind, long off) {
  dd v;
  if (kind == 0) ld_real(reinterpret_cast<const double *>(base) + off, v);
  else if (kind == 1) ld_real(reinterpret_cast<const dd *>(base) + off, v);
  else { v.hi = reinterpret_cast<const float *>(base)[off]; v.lo = 0.f; }
  return v;
}
template <>
__device__ __forceinline__ float ld_in<PolF>(const void *base, int kind, long off) {
  float v;
  if (kind == 0) ld_real(reinterpret_cast<const double *>(base) + off, v);
  else if (kind == 1) { const dd *p = reinterpret_cast<const dd *>(base) + off; v = __fadd_rn(p->hi, p->lo); }
  else v = reinterpret_cast<const float *>(base)[off];
  return v;
}
template <>
__device__ __forceinline__ double ld_in<PolD>(const void *base, int kind, long off) {
  if (kind == 0) return reinterpret_cast<const double *>(base)[off];
  if (kind == 1) return dd_to_double(reinterpret_cast<const dd *>(base)[off]);
  return (double)reinterpret_cast<const float *>(base)[off];
}
template <class P>
__device__ __forceinline__ void st_out(void *base, int kind, long off, typename P::re v);
template <>
__device__ __forceinline__ void st_out<PolD>(void *base, int kind, long off, double v) {
  if (kind == 0) reinterpret_cast<double *>(base)[off] = v;
  else if (kind == 1) reinterpret_cast<dd *>(base)[off] = dd_from_double(v);
  else reinterpret_cast<float *>(base)[off] = __double2float_rn(v);
}
template <>
__device__ __forceinline__ void st_out<PolDD>(void *base, int kind, long off, dd v) {
  if (kind == 0) st_real(reinterpret_cast<double *>(base) + off, v);
  else if (kind == 1) st_real(reinterpret_cast<dd *>(base) + off, v);
  else reinterpret_cast<float *>(base)[off] = __fadd_rn(v.hi, v.lo);
}
template <>
__device__ __forceinline__ void st_out<PolF>(void *base, int kind, long off, float v) {
  if (kind == 0) st_real(reinterpret_cast<double *>(base) + off, v);
  else if (kind == 1) { dd t; t.hi = v; t.lo = 0.f; st_real(reinterpret_cast<dd *>(base) + off, t); }
  else reinterpret_cast<float *>(base)[off] = v;
}

// y[off] += v (the prior's accumulate mode; double and dd outputs)
template <class P>
__device__ __forceinline__ void add_out(void *base, int kind, long off, typename P::re v);
template <>
__device__ __forceinline__ void add_out<PolDD>(void *base, int kind, long off, dd v) {
  if (kind == 0) {
    double *p = reinterpret_cast<double *>(base) + off;
    *p = *p + dd_to_double(v);
  } else if (kind == 1) {
    dd *p = reinterpret_cast<dd *>(base) + off;
    *p = dd_add(*p, v);
  } else {
    float *p = reinterpret_cast<float *>(base) + off;
    *p = *p + __fadd_rn(v.hi, v.lo);
  }
}
template <>
__device__ __forceinline__ void add_out<PolF>(void *base, int kind, long off, float v) {
  if (kind == 0) { double *p = reinterpret_cast<double *>(base) + off; *p = *p + (double)v; }
  else if (kind == 1) { dd *p = reinterpret_cast<dd *>(base) + off; dd t; t.hi = v; t.lo = 0.f; *p = dd_add(*p, t); }
  else { float *p = reinterpret_cast<float *>(base) + off; *p = *p + v; }
}
template <>
__device__ __forceinline__ void add_out<PolD>(void *base, int kind, long off, double v) {
  if (kind == 0) { double *p = reinterpret_cast<double *>(base) + off; *p = *p + v; }
}

// --------------------------------------------------------- time axis
// buf[k B + b] = in[k ld + n0 + b] for k < nk, b < B (zero where n0 + b >= N),
// every element copied asynchronously (cp.async, zero-filled past N) so that
// a thread's loads are all in flight at once; the caller's __syncthreads()
// after this makes the tile visible to the CTA
template <class P>
__device__ __forceinline__ void stage_cols(typename P::cx *buf, const typename P::cx *in, long ld,
                                           long n0, long N, int nk, int B) {
  constexpr int SZ = (int)sizeof(typename P::cx);
  static_assert(SZ == 8 || SZ == 16, "cp.async copies 8 or 16 bytes");
  for (int idx = threadIdx.x; idx < nk * B; idx += blockDim.x) {
    const int b = idx % B, k = idx / B;
    const long n = n0 + b;
    const bool ok = n < N;
    const typename P::cx *src = ok ? in + (long)k * ld + n : in;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(buf + idx);
    if (SZ == 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

template <class P>
__global__ void __launch_bounds__(256, P::occ)
k_rfft_time(const void *__restrict__ in, int in_kind, long in_ld, int n_in,
            typename P::cx *__restrict__ out, long out_ld, int N, FftPlan pl,
            const typename P::cx *__restrict__ twM, const typename P::cx *__restrict__ twL,
            int B, BatchArg ba) {
  typedef typename P::cx cx;
  typedef typename P::re re;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = pl.M;
  cx *buf0 = reinterpret_cast<cx *>(smem_raw);
  cx *buf1 = buf0 + (M + 1) * B;
  const long n0 = (long)blockIdx.x * B;
  const int bz = blockIdx.y;
  const int nin = min(ba.window(bz, n_in), M);
  const long ioff = bz * ba.in_stride;
  out += bz * ba.out_stride;
  // pack z_j = x_{2j} + i x_{2j+1}; x_t = 0 for t >= nin
  for (int idx = threadIdx.x; idx < M * B; idx += blockDim.x) {
    const int b = idx % B, j = idx / B;
    const long n = n0 + b;
    re r = P::re_zero(), im = P::re_zero();
    if (n < N) {
      const int t0 = 2 * j, t1 = 2 * j + 1;
      if (t0 < nin) r = ld_in<P>(in, in_kind, ioff + (long)t0 * in_ld + n);
      if (t1 < nin) im = ld_in<P>(in, in_kind, ioff + (long)t1 * in_ld + n);
    }
    buf0[j * B + b] = P::make(r, im);
  }
  __syncthreads();
  cx *Z = fft_run<P, false>(buf0, buf1, twM, pl, B, B, 1, true);
  // X_k = (Z_k + conj Z_{M-k})/2 + W_L^k (Z_k - conj Z_{M-k})/(2i)
  for (int idx = threadIdx.x; idx < (M + 1) * B; idx += blockDim.x) {
    const int b = idx % B, k = idx / B;
    const long n = n0 + b;
    if (n >= N) continue;
    cx zk = Z[(k % M) * B + b];
    cx zc = P::conj(Z[((M - k) % M) * B + b]);
    cx E = P::scale2(P::add(zk, zc), 0.5f);
    cx O = P::scale2(P::mul_mi(P::sub(zk, zc)), 0.5f);
    cx X = P::add(E, P::mul(ld_cx<P>(twL + k), O));
    out[(long)k * out_ld + n] = X;
  }
}

template <class P>
__global__ void __launch_bounds__(256, P::occ)
k_irfft_time(const typename P::cx *__restrict__ in, long in_ld, void *__restrict__ out,
             int out_kind, long out_ld, int N, int n_keep, FftPlan pl,
             const typename P::cx *__restrict__ twM, const typename P::cx *__restrict__ twL,
             typename P::re invM, int B, BatchArg ba) {
  typedef typename P::cx cx;
  typedef typename P::re re;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = pl.M;
  cx *buf0 = reinterpret_cast<cx *>(smem_raw);
  cx *buf1 = buf0 + (M + 1) * B;
  const long n0 = (long)blockIdx.x * B;
  const int bz = blockIdx.y;
  in += bz * ba.in_stride;
  const long ooff = bz * ba.out_stride;
  const int nkeep = ba.window(bz, n_keep);
  stage_cols<P>(buf0, in, in_ld, n0, N, M + 1, B);
  __syncthreads();
  // Z_k = E_k + i O_k, E_k = (X_k + conj X_{M-k})/2, O_k = (X_k - conj X_{M-k}) W_L^{-k} / 2
  for (int idx = threadIdx.x; idx < M * B; idx += blockDim.x) {
    const int b = idx % B, k = idx / B;
    cx xk = buf0[k * B + b];
    cx xc = P::conj(buf0[(M - k) * B + b]);
    cx E = P::scale2(P::add(xk, xc), 0.5f);
    cx O = P::scale2(P::mul(P::sub(xk, xc), P::conj(ld_cx<P>(twL + k))), 0.5f);
    buf1[k * B + b] = P::add(E, P::mul_i(O));
  }
  __syncthreads();
  cx *z = fft_run<P, true>(buf1, buf0, twM, pl, B, B, 1, true);
  for (int idx = threadIdx.x; idx < M * B; idx += blockDim.x) {
    const int b = idx % B, t = idx / B;
    const long n = n0 + b;
    if (n >= N) continue;
    re v = P::re_zero();
    if (t < nkeep) {
      cx zz = z[(t >> 1) * B + b];
      v = P::re_mul((t & 1) ? P::imag(zz) : P::real(zz), invM);
    }
    st_out<P>(out, out_kind, ooff + (long)t * out_ld + n, v);
  }
}

// Inverse transform of a parameter spectrum (x^ -> m, truncated to the
// window, written to `out`) followed in shared memory by the forward
// transform of m (-> m^ into `spec`, which may be `in`: a CTA reads all of its
// columns before it writes them).  The forecast's time FFT of m then needs no
// second pass over m in HBM and no conversion of m back from its stored type.
template <class P>
__global__ void __launch_bounds__(256, P::occ)
k_irfft_rfft_time(const typename P::cx *in, long in_ld, void *__restrict__ out, int out_kind,
                  long out_ld, typename P::cx *spec, long spec_ld, int N, int n_keep_all, FftPlan pl,
                  const typename P::cx *__restrict__ twM, const typename P::cx *__restrict__ twL,
                  typename P::re invM, int B, BatchArg ba) {
  typedef typename P::cx cx;
  typedef typename P::re re;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // right-hand side bz: spectrum at in / spec + bz * (in_stride / work_stride),
  // m at out + bz * out_stride, its own window
  const int bz = blockIdx.y;
  in += bz * ba.in_stride;
  spec += bz * ba.work_stride;
  const long ooff = bz * ba.out_stride;
  const int n_keep = ba.window(bz, n_keep_all);
  const int M = pl.M;
  cx *buf0 = reinterpret_cast<cx *>(smem_raw);
  cx *buf1 = buf0 + (M + 1) * B;
  const long n0 = (long)blockIdx.x * B;
  stage_cols<P>(buf0, in, in_ld, n0, N, M + 1, B);
  __syncthreads();
  // inverse: Z_k = E_k + i O_k (as in k_irfft_time)
  for (int idx = threadIdx.x; idx < M * B; idx += blockDim.x) {
    const int b = idx % B, k = idx / B;
    cx xk = buf0[k * B + b];
    cx xc = P::conj(buf0[(M - k) * B + b]);
    cx E = P::scale2(P::add(xk, xc), 0.5f);
    cx O = P::scale2(P::mul(P::sub(xk, xc), P::conj(ld_cx<P>(twL + k))), 0.5f);
    buf1[k * B + b] = P::add(E, P::mul_i(O));
  }
  __syncthreads();
  cx *z = fft_run<P, true>(buf1, buf0, twM, pl, B, B, 1, true);
  cx *w = z == buf0 ? buf1 : buf0;
  // m_t = invM (Re, Im) z_{t/2} for t < n_keep, else 0: written out, and
  // packed again as the forward transform's input m_{2j} + i m_{2j+1}
  for (int idx = threadIdx.x; idx < M * B; idx += blockDim.x) {
    const int b = idx % B, j = idx / B;
    const long n = n0 + b;
    const cx zz = z[j * B + b];
    const int t0 = 2 * j, t1 = 2 * j + 1;
    re r0 = P::re_zero(), r1 = P::re_zero();
    if (t0 < n_keep) r0 = P::re_mul(P::real(zz), invM);
    if (t1 < n_keep) r1 = P::re_mul(P::imag(zz), invM);
    // the padded transform of length 2M holds m_t for t < M only
    if (n < N) {
      if (t0 < M) st_out<P>(out, out_kind, ooff + (long)t0 * out_ld + n, r0);
      if (t1 < M) st_out<P>(out, out_kind, ooff + (long)t1 * out_ld + n, r1);
    }
    w[j * B + b] = P::make(t0 < M ? r0 : P::re_zero(), t1 < M ? r1 : P::re_zero());
  }
  __syncthreads();
  cx *Z = fft_run<P, false>(w, z, twM, pl, B, B, 1, true);
  // X_k = (Z_k + conj Z_{M-k})/2 + W_L^k (Z_k - conj Z_{M-k})/(2i)  (as in k_rfft_time)
  for (int idx = threadIdx.x; idx < (M + 1) * B; idx += blockDim.x) {
    const int b = idx % B, k = idx / B;
    const long n = n0 + b;
    if (n >= N) continue;
    cx zk = Z[(k % M) * B + b];
    cx zc = P::conj(Z[((M - k) % M) * B + b]);
    cx E = P::scale2(P::add(zk, zc), 0.5f);
    cx O = P::scale2(P::mul_mi(P::sub(zk, zc)), 0.5f);
    spec[(long)k * spec_ld + n] = P::add(E, P::mul(ld_cx<P>(twL + k), O));
  }
}

// ------------------------------------------------------- Matern filter
// output field of input field t: (t / per) * stride + off + t % per
struct FieldMap {
  int per, stride, off;
  __device__ __forceinline__ long operator()(int t) const {
    return (long)(t / per) * stride + off + t % per;
  }
};

// rows pass: pair tp holds z = x_{2tp} + i x_{2tp+1}; FFT along b (length Ny)
template <class P, bool INV>
__global__ void __launch_bounds__(256, P::occ)
k_prior_rows(const void *__restrict__ x, int in_kind, void *__restrict__ y, int out_kind,
             typename P::cx *__restrict__ work, int nt, int Nx, int Ny, FftPlan ply,
             const typename P::cx *__restrict__ twy, int BR, FieldMap fm, BatchArg ba, int accum) {
  typedef typename P::cx cx;
  typedef typename P::re re;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx *buf0 = reinterpret_cast<cx *>(smem_raw);
  cx *buf1 = buf0 + BR * Ny;
  const int tp = blockIdx.y;
  const int a0 = blockIdx.x * BR;
  const int t0 = 2 * tp, t1 = 2 * tp + 1;
  const int bz = blockIdx.z;
  // fields t >= ntb of this batch entry are zero (input) / written as zero
  const int ntb = ba.window(bz, nt);
  const long xoff = bz * ba.in_stride, yoff = bz * ba.out_stride;
  work += bz * ba.work_stride;
  if (t0 >= ntb) {
    if (INV && !accum) {
      for (int idx = threadIdx.x; idx < BR * Ny; idx += blockDim.x) {
        const int j = idx % Ny, b = idx / Ny, a = a0 + b;
        if (a >= Nx) continue;
        st_out<P>(y, out_kind, yoff + ((long)fm(t0) * Nx + a) * Ny + j, P::re_zero());
        if (t1 < nt) st_out<P>(y, out_kind, yoff + ((long)fm(t1) * Nx + a) * Ny + j, P::re_zero());
      }
    }
    return;
  }
  for (int idx = threadIdx.x; idx < BR * Ny; idx += blockDim.x) {
    const int j = idx % Ny, b = idx / Ny, a = a0 + b;
    cx v = P::zero();
    if (a < Nx) {
      if (!INV) {
        re r = ld_in<P>(x, in_kind, xoff + ((long)t0 * Nx + a) * Ny + j);
        re im = (t1 < ntb) ? ld_in<P>(x, in_kind, xoff + ((long)t1 * Nx + a) * Ny + j) : P::re_zero();
        v = P::make(r, im);
      } else {
        v = work[((long)tp * Nx + a) * Ny + j];
      }
    }
    buf0[b * Ny + j] = v;
  }
  __syncthreads();
  cx *Z = fft_run<P, INV>(buf0, buf1, twy, ply, BR, 1, Ny, false);
  for (int idx = threadIdx.x; idx < BR * Ny; idx += blockDim.x) {
    const int j = idx % Ny, b = idx / Ny, a = a0 + b;
    if (a >= Nx) continue;
    cx v = Z[b * Ny + j];
    if (!INV) {
      work[((long)tp * Nx + a) * Ny + j] = v;
    } else {
      const long o0 = yoff + ((long)fm(t0) * Nx + a) * Ny + j;
      const long o1 = yoff + ((long)fm(t1) * Nx + a) * Ny + j;
      if (accum) {
        add_out<P>(y, out_kind, o0, P::real(v));
        if (t1 < ntb) add_out<P>(y, out_kind, o1, P::imag(v));
      } else {
        st_out<P>(y, out_kind, o0, P::real(v));
        if (t1 < nt) st_out<P>(y, out_kind, o1, t1 < ntb ? P::imag(v) : P::re_zero());
      }
    }
  }
}

// columns pass: forward FFT along a (length Nx, stride Ny), scale by lambda,
// inverse FFT along a, in place in `work`.
template <class P>
__global__ void __launch_bounds__(256, P::occ)
k_prior_cols(typename P::cx *__restrict__ work, const typename P::re *__restrict__ lam, int Nx,
             int Ny, FftPlan plx, const typename P::cx *__restrict__ twx, int BC, int nt,
             BatchArg ba) {
  typedef typename P::cx cx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx *buf0 = reinterpret_cast<cx *>(smem_raw);
  cx *buf1 = buf0 + Nx * BC;
  const int tp = blockIdx.y;
  const int j0 = blockIdx.x * BC;
  const int bz = blockIdx.z;
  if (2 * tp >= ba.window(bz, nt)) return;
  cx *wp = work + bz * ba.work_stride + (long)tp * Nx * Ny;
  for (int idx = threadIdx.x; idx < Nx * BC; idx += blockDim.x) {
    const int b = idx % BC, a = idx / BC, j = j0 + b;
    buf0[a * BC + b] = (j < Ny) ? wp[(long)a * Ny + j] : P::zero();
  }
  __syncthreads();
  cx *Z = fft_run<P, false>(buf0, buf1, twx, plx, BC, BC, 1, true);
  cx *O = (Z == buf0) ? buf1 : buf0;
  for (int idx = threadIdx.x; idx < Nx * BC; idx += blockDim.x) {
    const int b = idx % BC, p = idx / BC, j = j0 + b;
    if (j < Ny) Z[p * BC + b] = P::scale_re(Z[p * BC + b], lam[(long)p * Ny + j]);
  }
  __syncthreads();
  cx *Y = fft_run<P, true>(Z, O, twx, plx, BC, BC, 1, true);
  for (int idx = threadIdx.x; idx < Nx * BC; idx += blockDim.x) {
    const int b = idx % BC, a = idx / BC, j = j0 + b;
    if (j < Ny) wp[(long)a * Ny + j] = Y[a * BC + b];
  }
}

// Complex fields, FP64 (set-up): rows pass of C applied to x[f] (cdd storage)
// for fields f in [0, nf); forward: x -> work (cd), inverse: work -> x.
template <bool INV>
__global__ void __launch_bounds__(256)
k_cfield_rows(cdd *__restrict__ x, cd *__restrict__ work, int Nx, int Ny, FftPlan ply,
              const cd *__restrict__ twy, int BR) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cd *buf0 = reinterpret_cast<cd *>(smem_raw);
  cd *buf1 = buf0 + BR * Ny;
  const int f = blockIdx.y, a0 = blockIdx.x * BR;
  cdd *xf = x + (long)f * Nx * Ny;
  cd *wf = work + (long)f * Nx * Ny;
  for (int idx = threadIdx.x; idx < BR * Ny; idx += blockDim.x) {
    const int j = idx % Ny, b = idx / Ny, a = a0 + b;
    cd v = PolD::zero();
    if (a < Nx) {
      if (!INV) {
        const cdd z = ld_cdd(xf + (long)a * Ny + j);
        v = PolD::make(dd_to_double(z.re), dd_to_double(z.im));
      } else {
        v = wf[(long)a * Ny + j];
      }
    }
    buf0[b * Ny + j] = v;
  }
  __syncthreads();
  cd *Z = fft_run<PolD, INV>(buf0, buf1, twy, ply, BR, 1, Ny, false);
  for (int idx = threadIdx.x; idx < BR * Ny; idx += blockDim.x) {
    const int j = idx % Ny, b = idx / Ny, a = a0 + b;
    if (a >= Nx) continue;
    const cd v = Z[b * Ny + j];
    if (!INV) {
      wf[(long)a * Ny + j] = v;
    } else {
      cdd z;
      z.re = dd_from_double(v.re);
      z.im = dd_from_double(v.im);
      st_cdd(xf + (long)a * Ny + j, z);
    }
  }
}

template <class KER>
void ensure_smem(KER k, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int pick_batch(int len, size_t elem, int cap, size_t budget) {
  // two ping-pong buffers of len x B elements within the budget
  int B = 1;
  while (B * 2 <= cap && (size_t)2 * len * (B * 2) * elem <= budget) B *= 2;
  return B;
}

template <class P>
cudaError_t rfft_time(const void *in, int in_kind, long in_ld, int n_in, typename P::cx *out,
                      long out_ld, int N, const FftPlan &pl, const typename P::cx *twM,
                      const typename P::cx *twL, cudaStream_t s, BatchArg ba = BatchArg{}) {
  if (N <= 0 || ba.count <= 0) return cudaSuccess;
  const int B = pick_batch(pl.M + 1, sizeof(typename P::cx), 32, P::smem);
  const size_t sm = (size_t)2 * (pl.M + 1) * B * sizeof(typename P::cx);
  ensure_smem(k_rfft_time<P>, sm);
  const dim3 grid((unsigned)((N + B - 1) / B), (unsigned)ba.count);
  k_rfft_time<P><<<grid, 256, sm, s>>>(in, in_kind, in_ld, n_in, out, out_ld, N, pl, twM, twL, B,
                                       ba);
  count_launches(1);
  return cudaGetLastError();
}

template <class P>
cudaError_t irfft_time(const typename P::cx *in, long in_ld, void *out, int out_kind, long out_ld,
                       int N, int n_keep, const FftPlan &pl, const typename P::cx *twM,
                       const typename P::cx *twL, typename P::re invM, cudaStream_t s,
                       BatchArg ba = BatchArg{}) {
  if (N <= 0 || ba.count <= 0) return cudaSuccess;
  const int B = pick_batch(pl.M + 1, sizeof(typename P::cx), 32, P::smem);
  const size_t sm = (size_t)2 * (pl.M + 1) * B * sizeof(typename P::cx);
  ensure_smem(k_irfft_time<P>, sm);
  const dim3 grid((unsigned)((N + B - 1) / B), (unsigned)ba.count);
  k_irfft_time<P><<<grid, 256, sm, s>>>(in, in_ld, out, out_kind, out_ld, N, n_keep, pl, twM, twL,
                                        invM, B, ba);
  count_launches(1);
  return cudaGetLastError();
}

template <class P>
cudaError_t prior(const void *x, int in_kind, void *y, int out_kind, int nt, int Nx, int Ny,
                  typename P::cx *work, const typename P::re *lam, const FftPlan &plx,
                  const FftPlan &ply, const typename P::cx *twx, const typename P::cx *twy,
                  cudaStream_t s, FieldMap fm = FieldMap{1 << 30, 0, 0}, BatchArg ba = BatchArg{},
                  int accum = 0) {
  if (nt <= 0 || ba.count <= 0) return cudaSuccess;
  typedef typename P::cx cx;
  const int np = (nt + 1) / 2;
  int BR = 1;
  while (BR * 2 <= 16 && (size_t)2 * (BR * 2) * Ny * sizeof(cx) <= (size_t)P::smem) BR *= 2;
  int BC = 1;
  while (BC * 2 <= 16 && (size_t)2 * (BC * 2) * Nx * sizeof(cx) <= (size_t)P::smem) BC *= 2;
  const size_t smr = (size_t)2 * BR * Ny * sizeof(cx);
  const size_t smc = (size_t)2 * BC * Nx * sizeof(cx);
  ensure_smem(k_prior_rows<P, false>, smr);
  ensure_smem(k_prior_rows<P, true>, smr);
  ensure_smem(k_prior_cols<P>, smc);
  dim3 gr((Nx + BR - 1) / BR, np, ba.count), gc((Ny + BC - 1) / BC, np, ba.count);
  k_prior_rows<P, false><<<gr, 256, smr, s>>>(x, in_kind, nullptr, 0, work, nt, Nx, Ny, ply, twy, BR,
                                              fm, ba, 0);
  count_launches(1);
  k_prior_cols<P><<<gc, 256, smc, s>>>(work, lam, Nx, Ny, plx, twx, BC, nt, ba);
  count_launches(1);
  k_prior_rows<P, true><<<gr, 256, smr, s>>>(nullptr, 0, y, out_kind, work, nt, Nx, Ny, ply, twy, BR,
                                             fm, ba, accum);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rfft_time_dd(const void *in, int in_kind, long in_ld, int n_in, cdd *out,
                                long out_ld, int N, const FftPlan &pl, const cdd *twM,
                                const cdd *twL, cudaStream_t s, const BatchArg &ba) {
  return rfft_time<PolDD>(in, in_kind, in_ld, n_in, out, out_ld, N, pl, twM, twL, s, ba);
}
cudaError_t launch_rfft_time_f(const void *in, int in_kind, long in_ld, int n_in, cf *out,
                               long out_ld, int N, const FftPlan &pl, const cf *twM,
                               const cf *twL, cudaStream_t s, const BatchArg &ba) {
  return rfft_time<PolF>(in, in_kind, in_ld, n_in, out, out_ld, N, pl, twM, twL, s, ba);
}
template <class P>
cudaError_t irfft_rfft_time(const typename P::cx *in, long in_ld, void *out, int out_kind, long out_ld,
                            typename P::cx *spec, long spec_ld, int N, int n_keep, const FftPlan &pl,
                            const typename P::cx *twM, const typename P::cx *twL, typename P::re invM,
                            cudaStream_t s, const BatchArg &ba) {
  if (N <= 0 || ba.count <= 0) return cudaSuccess;
  const int B = pick_batch(pl.M + 1, sizeof(typename P::cx), 32, P::smem);
  const size_t sm = (size_t)2 * (pl.M + 1) * B * sizeof(typename P::cx);
  ensure_smem(k_irfft_rfft_time<P>, sm);
  const dim3 grid((unsigned)((N + B - 1) / B), (unsigned)ba.count);
  k_irfft_rfft_time<P><<<grid, 256, sm, s>>>(in, in_ld, out, out_kind, out_ld, spec, spec_ld, N, n_keep, pl,
                                             twM, twL, invM, B, ba);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_irfft_rfft_time_dd(const cdd *in, long in_ld, void *out, int out_kind, long out_ld,
                                      cdd *spec, long spec_ld, int N, int n_keep, const FftPlan &pl,
                                      const cdd *twM, const cdd *twL, cudaStream_t s, const BatchArg &ba) {
  const double inv = 1.0 / pl.M;
  dd invM;
  invM.hi = (float)inv;
  invM.lo = (float)(inv - (double)invM.hi);
  return irfft_rfft_time<PolDD>(in, in_ld, out, out_kind, out_ld, spec, spec_ld, N, n_keep, pl, twM, twL,
                                invM, s, ba);
}
cudaError_t launch_irfft_rfft_time_f(const cf *in, long in_ld, void *out, int out_kind, long out_ld,
                                     cf *spec, long spec_ld, int N, int n_keep, const FftPlan &pl,
                                     const cf *twM, const cf *twL, cudaStream_t s, const BatchArg &ba) {
  return irfft_rfft_time<PolF>(in, in_ld, out, out_kind, out_ld, spec, spec_ld, N, n_keep, pl, twM, twL,
                               (float)(1.0 / pl.M), s, ba);
}
cudaError_t launch_irfft_time_dd(const cdd *in, long in_ld, void *out, int out_kind, long out_ld,
                                 int N, int n_keep, const FftPlan &pl, const cdd *twM,
                                 const cdd *twL, cudaStream_t s, const BatchArg &ba) {
  // 1/M as a float pair (host double split)
  const double inv = 1.0 / pl.M;
  dd invM;
  invM.hi = (float)inv;
  invM.lo = (float)(inv - (double)invM.hi);
  return irfft_time<PolDD>(in, in_ld, out, out_kind, out_ld, N, n_keep, pl, twM, twL, invM, s, ba);
}
cudaError_t launch_irfft_time_f(const cf *in, long in_ld, void *out, int out_kind, long out_ld,
                                int N, int n_keep, const FftPlan &pl, const cf *twM,
                                const cf *twL, cudaStream_t s, const BatchArg &ba) {
  return irfft_time<PolF>(in, in_ld, out, out_kind, out_ld, N, n_keep, pl, twM, twL,
                          (float)(1.0 / pl.M), s, ba);
}
cudaError_t launch_prior_dd(const void *x, int in_kind, void *y, int out_kind, int nt, int Nx,
                            int Ny, cdd *work, const dd *lam, const FftPlan &plx,
                            const FftPlan &ply, const cdd *twx, const cdd *twy, cudaStream_t s,
                            const BatchArg &ba, int accum) {
  return prior<PolDD>(x, in_kind, y, out_kind, nt, Nx, Ny, work, lam, plx, ply, twx, twy, s,
                      FieldMap{1 << 30, 0, 0}, ba, accum);
}
cudaError_t launch_prior_d(const void *x, int in_kind, void *y, int out_kind, int nt, int Nx,
                           int Ny, cd *work, const double *lam, const FftPlan &plx,
                           const FftPlan &ply, const cd *twx, const cd *twy, int map_per,
                           int map_stride, int map_off, cudaStream_t s) {
  return prior<PolD>(x, in_kind, y, out_kind, nt, Nx, Ny, work, lam, plx, ply, twx, twy, s,
                     FieldMap{map_per, map_stride, map_off});
}
// x[f] <- C x[f] for complex fields f < nf (cdd storage, FP64 arithmetic);
// lam: eigenvalues / (Nx Ny) in FP64; work: nf_chunk fields of cd
cudaError_t launch_prior_cfields_d(cdd *x, long nf, int Nx, int Ny, cd *work, long nf_chunk,
                                   const double *lam, const FftPlan &plx, const FftPlan &ply,
                                   const cd *twx, const cd *twy, cudaStream_t s) {
  int BR = 1;
  while (BR * 2 <= 16 && (size_t)2 * (BR * 2) * Ny * sizeof(cd) <= 64 * 1024) BR *= 2;
  int BC = 1;
  while (BC * 2 <= 16 && (size_t)2 * (BC * 2) * Nx * sizeof(cd) <= 64 * 1024) BC *= 2;
  const size_t smr = (size_t)2 * BR * Ny * sizeof(cd), smc = (size_t)2 * BC * Nx * sizeof(cd);
  ensure_smem(k_cfield_rows<false>, smr);
  ensure_smem(k_cfield_rows<true>, smr);
  ensure_smem(k_prior_cols<PolD>, smc);
  for (long f0 = 0; f0 < nf; f0 += nf_chunk) {
    const int nc = (int)std::min<long>(nf_chunk, nf - f0);
    cdd *xc = x + f0 * Nx * Ny;
    dim3 gr((Nx + BR - 1) / BR, nc), gc((Ny + BC - 1) / BC, nc);
    k_cfield_rows<false><<<gr, 256, smr, s>>>(xc, work, Nx, Ny, ply, twy, BR);
    k_prior_cols<PolD><<<gc, 256, smc, s>>>(work, lam, Nx, Ny, plx, twx, BC, 2 * nc, BatchArg{});
    k_cfield_rows<true><<<gr, 256, smr, s>>>(xc, work, Nx, Ny, ply, twy, BR);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_prior_f(const void *x, int in_kind, void *y, int out_kind, int nt, int Nx,
                           int Ny, cf *work, const float *lam, const FftPlan &plx,
                           const FftPlan &ply, const cf *twx, const cf *twy, cudaStream_t s,
                           const BatchArg &ba, int accum) {
  return prior<PolF>(x, in_kind, y, out_kind, nt, Nx, Ny, work, lam, plx, ply, twx, twy, s,
                     FieldMap{1 << 30, 0, 0}, ba, accum);
}

}  // namespace tw
