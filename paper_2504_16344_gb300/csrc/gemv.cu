// gemv.cu -- one complex matrix-vector product per frequency.
//
// After the time FFT the block Toeplitz apply is block diagonal in frequency
// (Sec. "FFT-based Hessian matvecs"): y^(w) = F^(w) x^(w) for the forward
// map and x^(w) = F^(w)^H y^(w) for the adjoint, w = 0..Nt.  The operator
// F^ ([Nf][Nr][Nm], Nr = Nd or Nq rows, grid index contiguous) is streamed
// exactly once per apply; this is the HBM-bound step.
//
//  * adjoint: a thread owns KPT grid points k and walks the Nr rows, so the
//    per-k sums need no cross-thread reduction; y^(w) sits in shared memory.
//  * forward: a CTA owns one frequency and a chunk of 32*JPL grid points
//    (x^ chunk in shared memory); each warp takes whole rows, every lane sums
//    JPL products, a shuffle tree reduces the warp, and the per-chunk partial
//    sums are added by a second small kernel in a fixed order.
//
// The FP64-class path reads float-pair entries (16 B) and accumulates with
// exact products and a compensated running sum; the reduced-precision
// paths read complex64 or bf16 hi+lo entries (8 B): the forward product
// sums in FP32; the adjoint of one right-hand side forms exact products and
// a double-float running sum (several right-hand sides: gemm_sl.cu).
#include "kernels.h"

namespace tw {

namespace {

constexpr int ADJ_KPT = 4;     // grid points per thread (adjoint)
constexpr int FWD_JPL = 32;    // grid points per lane per row (forward)
constexpr int FWD_KC = 32 * FWD_JPL;

__device__ __forceinline__ float4 ld_stream4(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream2(const float2 *p) { return __ldcs(p); }
__device__ __forceinline__ uint2 ld_stream_u2(const uint2 *p) { return __ldcs(p); }

__device__ __forceinline__ float bf16lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }

// complex entry of an FP32-path operator: C64 (float2) or BF16X2 (re_hi, re_lo, im_hi, im_lo)
template <int FMT>
__device__ __forceinline__ cf ld_op_f(const void *A, size_t i);
template <>
__device__ __forceinline__ cf ld_op_f<FMT_C64>(const void *A, size_t i) {
  float2 v = ld_stream2(reinterpret_cast<const float2 *>(A) + i);
  return cf_make(v.x, v.y);
}
template <>
__device__ __forceinline__ cf ld_op_f<FMT_BF16X2>(const void *A, size_t i) {
  uint2 v = ld_stream_u2(reinterpret_cast<const uint2 *>(A) + i);
  // low half of each word = hi part, high half = lo part
  return cf_make(bf16lo(v.x) + bf16hi(v.x), bf16lo(v.y) + bf16hi(v.y));
}

// ------------------------------------------------------------ adjoint
__global__ void __launch_bounds__(256)
k_gemv_adj_dd(const float4 *__restrict__ A, const cdd *__restrict__ yh, cdd *__restrict__ xh,
              int Nr, int Nm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cdd *sy = reinterpret_cast<cdd *>(smem_raw);
  const int w = blockIdx.y;
  const float4 *Aw = A + (size_t)w * Nr * Nm;
  for (int s = threadIdx.x; s < Nr; s += blockDim.x) sy[s] = ld_cdd(yh + (size_t)w * Nr + s);
  __syncthreads();
  const int kb = blockIdx.x * (256 * ADJ_KPT) + threadIdx.x;
  // Nr (<= a few hundred) terms per sum: the renormalised accumulator
  // needs no extra folding here (it would only cost registers)
  dacc re[ADJ_KPT], im[ADJ_KPT];
  bool ok[ADJ_KPT];
#pragma unroll
  for (int j = 0; j < ADJ_KPT; ++j) {
    re[j] = dacc_zero(); im[j] = dacc_zero();
    ok[j] = kb + 256 * j < Nm;
  }
  float4 cur[ADJ_KPT], nxt[ADJ_KPT];
#pragma unroll
  for (int j = 0; j < ADJ_KPT; ++j)
    cur[j] = ok[j] ? ld_stream4(Aw + kb + 256 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int s = 0; s < Nr; ++s) {
    if (s + 1 < Nr) {
      const float4 *row = Aw + (size_t)(s + 1) * Nm + kb;
#pragma unroll
      for (int j = 0; j < ADJ_KPT; ++j) nxt[j] = ok[j] ? ld_stream4(row + 256 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const cdd y = sy[s];
#pragma unroll
    for (int j = 0; j < ADJ_KPT; ++j) {
      dd ar, ai;
      ar.hi = cur[j].x; ar.lo = cur[j].y; ai.hi = cur[j].z; ai.lo = cur[j].w;
      // conj(a) * y = (ar yr + ai yi) + i (ar yi - ai yr)
      dacc_mac(re[j], ar, y.re);
      dacc_mac(re[j], ai, y.im);
      dacc_mac(im[j], ar, y.im);
      dacc_mac(im[j], dd_neg(ai), y.re);
    }
#pragma unroll
    for (int j = 0; j < ADJ_KPT; ++j) cur[j] = nxt[j];
  }
#pragma unroll
  for (int j = 0; j < ADJ_KPT; ++j) {
    if (!ok[j]) continue;
    cdd r;
    r.re = dacc_get(re[j]);
    r.im = dacc_get(im[j]);
    st_cdd(xh + (size_t)w * Nm + kb + 256 * j, r);
  }
}

// ----------------------------------------- adjoint, FP32 operator, one RHS
// Reduced-precision adjoint for ONE right-hand side: the complex64 (or bf16
// hi+lo) operator times y's double-float spectrum, summed without rounding
// loss.  F^T y cancels (y = K^-1 d is large against m), so a plain FP32 sum
// of the terms would lose digits by that cancellation.  Each product of an
// operator entry a and y_hi is made exact (p + e = a y_hi by FMA), the large
// parts p are added to a running sum with TwoSum (Knuth) and the rounding
// errors, e, and the a y_lo terms are gathered in FP32 side sums: the result
// is the exact product of the rounded operator with y to about 2^-44 of the
// terms.  The real and imaginary parts of one grid point travel together in
// packed FP32 pairs (add/mul/fma.rn.f32x2), which halves the instruction
// count: the kernel streams the 8-byte operator at HBM speed.

// y row s as the packed operands of the kernel below: with yr, yi float pairs,
//   Y1 = (yr, yi)   (x ar -> the ar terms of Re, Im)
//   Y2 = (yi, -yr)  (x ai -> the ai terms)
// high parts, their negations (exact products via FMA) and low parts
struct AdjRow { f2 y1, y1n, y1l, y2, y2n, y2l; };

__device__ __forceinline__ void acc_two_sum(f2 &S, f2 &C, f2 pn) {
  // S + p with p = -pn: s = S - pn, exact error err = (S - (s - bb)) - (pn + bb)
  const f2 s = sub2(S, pn);
  const f2 bb = sub2(s, S);
  const f2 err = sub2(sub2(S, sub2(s, bb)), add2(pn, bb));
  S = s;
  C = add2(C, err);
}

template <int FMT>
__global__ void __launch_bounds__(256)
k_gemv_adj_cx(const void *__restrict__ A, const cdd *__restrict__ yh, cf *__restrict__ xh, int Nr,
              int Nm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AdjRow *sy = reinterpret_cast<AdjRow *>(smem_raw);
  const int w = blockIdx.y;
  const size_t base = (size_t)w * Nr * Nm;
  for (int s = threadIdx.x; s < Nr; s += blockDim.x) {
    const cdd y = ld_cdd(yh + (size_t)w * Nr + s);
    AdjRow r;
    r.y1 = f2_make(y.re.hi, y.im.hi);
    r.y1n = f2_make(-y.re.hi, -y.im.hi);
    r.y1l = f2_make(y.re.lo, y.im.lo);
    r.y2 = f2_make(y.im.hi, -y.re.hi);
    r.y2n = f2_make(-y.im.hi, y.re.hi);
    r.y2l = f2_make(y.im.lo, -y.re.lo);
    sy[s] = r;
  }
  __syncthreads();
  const int kb = blockIdx.x * (256 * ADJ_KPT) + threadIdx.x;
  f2 S[ADJ_KPT], C[ADJ_KPT], L[ADJ_KPT];
  bool ok[ADJ_KPT];
#pragma unroll
  for (int j = 0; j < ADJ_KPT; ++j) {
    S[j] = f2_make(0.f, 0.f); C[j] = S[j]; L[j] = S[j];
    ok[j] = kb + 256 * j < Nm;
  }
  // rows s+1 and s+2 in flight while row s is used (8-byte entries)
  cf cur[ADJ_KPT], nx1[ADJ_KPT], nx2[ADJ_KPT];
#pragma unroll
  for (int j = 0; j < ADJ_KPT; ++j) {
    cur[j] = ok[j] ? ld_op_f<FMT>(A, base + kb + 256 * j) : cf_zero();
    nx1[j] = (ok[j] && Nr > 1) ? ld_op_f<FMT>(A, base + (size_t)Nm + kb + 256 * j) : cf_zero();
  }
  for (int s = 0; s < Nr; ++s) {
    if (s + 2 < Nr) {
      const size_t row = base + (size_t)(s + 2) * Nm + kb;
#pragma unroll
      for (int j = 0; j < ADJ_KPT; ++j) nx2[j] = ok[j] ? ld_op_f<FMT>(A, row + 256 * j) : cf_zero();
    }
    const AdjRow y = sy[s];
#pragma unroll
    for (int j = 0; j < ADJ_KPT; ++j) {
      // conj(a) y = ar (yr, yi) + ai (yi, -yr)
      const f2 a1 = f2_make(cur[j].re, cur[j].re), a2 = f2_make(cur[j].im, cur[j].im);
      const f2 p1n = mul2(a1, y.y1n), p2n = mul2(a2, y.y2n);      // -(a y_hi), rounded
      const f2 e1 = fma2(a1, y.y1, p1n), e2 = fma2(a2, y.y2, p2n); // their exact errors
      acc_two_sum(S[j], C[j], p1n);
      acc_two_sum(S[j], C[j], p2n);
      L[j] = add2(fma2(a2, y.y2l, fma2(a1, y.y1l, L[j])), add2(e1, e2));
    }
#pragma unroll
    for (int j = 0; j < ADJ_KPT; ++j) { cur[j] = nx1[j]; nx1[j] = nx2[j]; }
  }
#pragma unroll
  for (int j = 0; j < ADJ_KPT; ++j) {
    if (!ok[j]) continue;
    const float2 r = f2_split(add2(S[j], add2(C[j], L[j])));
    xh[(size_t)w * Nm + kb + 256 * j] = cf_make(r.x, r.y);
  }
}

// ------------------------------------------------------------ forward
__device__ __forceinline__ dd shfl_xor_dd(dd v, int m) {
  dd r;
  r.hi = __shfl_xor_sync(0xffffffffu, v.hi, m);
  r.lo = __shfl_xor_sync(0xffffffffu, v.lo, m);
  return r;
}

__global__ void __launch_bounds__(256)
k_gemv_fwd_dd(const float4 *__restrict__ A, const cdd *__restrict__ xh, cdd *__restrict__ part,
              int Nr, int Nm, int nchunk) {
  __shared__ __align__(16) cdd sx[FWD_KC];
  const int w = blockIdx.y, c = blockIdx.x;
  const int kbase = c * FWD_KC;
  for (int i = threadIdx.x; i < FWD_KC; i += blockDim.x) {
    const int k = kbase + i;
    sx[i] = (k < Nm) ? ld_cdd(xh + (size_t)w * Nm + k) : cdd_zero();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvalid = min(FWD_KC, Nm - kbase);
  for (int s = warp; s < Nr; s += 8) {
    const float4 *row = A + ((size_t)w * Nr + s) * Nm + kbase;
    dacc re = dacc_zero(), im = dacc_zero();
    dd r = dd_zero(), i = dd_zero();
    for (int j0 = 0; j0 < FWD_JPL; j0 += 8) {
      // the group's eight loads are issued together, without a branch: past
      // the last grid point the index is clamped and x^ is zero there, so
      // those terms add exact zeros
      float4 a[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = ld_stream4(row + min(lane + 32 * (j0 + j), nvalid - 1));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const cdd x = sx[lane + 32 * (j0 + j)];
        dd ar, ai;
        ar.hi = a[j].x; ar.lo = a[j].y; ai.hi = a[j].z; ai.lo = a[j].w;
        dacc_mac(re, ar, x.re);
        dacc_mac(re, dd_neg(ai), x.im);
        dacc_mac(im, ar, x.im);
        dacc_mac(im, ai, x.re);
      }
      dacc_fold(r, re);
      dacc_fold(i, im);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      r = dd_add(r, shfl_xor_dd(r, m));
      i = dd_add(i, shfl_xor_dd(i, m));
    }
    if (lane == 0) {
      cdd o; o.re = r; o.im = i;
      st_cdd(part + ((size_t)w * nchunk + c) * Nr + s, o);
    }
  }
}

template <int FMT>
__global__ void __launch_bounds__(256)
k_gemv_fwd_f(const void *__restrict__ A, const cf *__restrict__ xh, cf *__restrict__ part, int Nr,
             int Nm, int nchunk) {
  __shared__ __align__(16) cf sx[FWD_KC];
  const int w = blockIdx.y, c = blockIdx.x;
  const int kbase = c * FWD_KC;
  for (int i = threadIdx.x; i < FWD_KC; i += blockDim.x) {
    const int k = kbase + i;
    sx[i] = (k < Nm) ? xh[(size_t)w * Nm + k] : cf_zero();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvalid = min(FWD_KC, Nm - kbase);
  for (int s = warp; s < Nr; s += 8) {
    const size_t row = ((size_t)w * Nr + s) * Nm + kbase;
    float re = 0.f, im = 0.f;
#pragma unroll 8
    for (int j = 0; j < FWD_JPL; ++j) {
      const int kk = lane + 32 * j;
      if (kk < nvalid) {
        const cf a = ld_op_f<FMT>(A, row + kk);
        const cf x = sx[kk];
        re = fmaf(a.re, x.re, fmaf(-a.im, x.im, re));
        im = fmaf(a.re, x.im, fmaf(a.im, x.re, im));
      }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, m);
      im += __shfl_xor_sync(0xffffffffu, im, m);
    }
    if (lane == 0) part[((size_t)w * nchunk + c) * Nr + s] = cf_make(re, im);
  }
}

__global__ void k_gemv_reduce_dd(const cdd *__restrict__ part, cdd *__restrict__ yh, int Nf,
                                 int Nr, int nchunk) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)Nf * Nr) return;
  const int w = (int)(idx / Nr), s = (int)(idx % Nr);
  dd re = dd_zero(), im = dd_zero();
  for (int c = 0; c < nchunk; ++c) {
    const cdd p = ld_cdd(part + ((size_t)w * nchunk + c) * Nr + s);
    re = dd_add(re, p.re);
    im = dd_add(im, p.im);
  }
  cdd o; o.re = re; o.im = im;
  st_cdd(yh + idx, o);
}

__global__ void k_gemv_reduce_f(const cf *__restrict__ part, cf *__restrict__ yh, int Nf, int Nr,
                                int nchunk) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)Nf * Nr) return;
  const int w = (int)(idx / Nr), s = (int)(idx % Nr);
  float re = 0.f, im = 0.f;
  for (int c = 0; c < nchunk; ++c) {
    const cf p = part[((size_t)w * nchunk + c) * Nr + s];
    re += p.re;
    im += p.im;
  }
  yh[idx] = cf_make(re, im);
}

// ------------------------------------------------------- conversion
__global__ void k_convert_op(const cdd *__restrict__ src, long src_ld_w, void *__restrict__ dst,
                             int fmt, long dst_ld_w, long n_per_w, int Nf) {
  const long total = (long)Nf * n_per_w;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const long w = idx / n_per_w, i = idx % n_per_w;
    const cdd v = ld_cdd(src + w * src_ld_w + i);
    const float re = __fadd_rn(v.re.hi, v.re.lo), im = __fadd_rn(v.im.hi, v.im.lo);
    if (fmt == FMT_C64) {
      reinterpret_cast<float2 *>(dst)[w * dst_ld_w + i] = make_float2(re, im);
    } else {
      const __nv_bfloat16 rh = __float2bfloat16_rn(re);
      const __nv_bfloat16 rl = __float2bfloat16_rn(re - __bfloat162float(rh));
      const __nv_bfloat16 ih = __float2bfloat16_rn(im);
      const __nv_bfloat16 il = __float2bfloat16_rn(im - __bfloat162float(ih));
      uint2 o;
      o.x = (unsigned)__bfloat16_as_ushort(rh) | ((unsigned)__bfloat16_as_ushort(rl) << 16);
      o.y = (unsigned)__bfloat16_as_ushort(ih) | ((unsigned)__bfloat16_as_ushort(il) << 16);
      reinterpret_cast<uint2 *>(dst)[w * dst_ld_w + i] = o;
    }
  }
}

}  // namespace

int gemv_fwd_nchunk(int Nm) { return (Nm + FWD_KC - 1) / FWD_KC; }

cudaError_t launch_gemv_fwd_dd(const void *A, int fmt, const cdd *xh, cdd *part, cdd *yh, int Nf,
                               int Nr, int Nm, cudaStream_t s) {
  if (fmt != FMT_DD) return cudaErrorInvalidValue;
  const int nchunk = gemv_fwd_nchunk(Nm);
  k_gemv_fwd_dd<<<dim3(nchunk, Nf), 256, 0, s>>>(reinterpret_cast<const float4 *>(A), xh, part,
                                                  Nr, Nm, nchunk);
  count_launches(1);
  const long n = (long)Nf * Nr;
  k_gemv_reduce_dd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, yh, Nf, Nr, nchunk);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gemv_fwd_f(const void *A, int fmt, const cf *xh, cf *part, cf *yh, int Nf,
                              int Nr, int Nm, cudaStream_t s) {
  const int nchunk = gemv_fwd_nchunk(Nm);
  if (fmt == FMT_C64)
    k_gemv_fwd_f<FMT_C64><<<dim3(nchunk, Nf), 256, 0, s>>>(A, xh, part, Nr, Nm, nchunk);
  else if (fmt == FMT_BF16X2)
    k_gemv_fwd_f<FMT_BF16X2><<<dim3(nchunk, Nf), 256, 0, s>>>(A, xh, part, Nr, Nm, nchunk);
  else
    return cudaErrorInvalidValue;
  count_launches(1);
  const long n = (long)Nf * Nr;
  k_gemv_reduce_f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, yh, Nf, Nr, nchunk);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gemv_adj_dd(const void *A, int fmt, const cdd *yh, cdd *xh, int Nf, int Nr,
                               int Nm, cudaStream_t s) {
  if (fmt != FMT_DD) return cudaErrorInvalidValue;
  const size_t sm = (size_t)Nr * sizeof(cdd);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_gemv_adj_dd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 g((Nm + 256 * ADJ_KPT - 1) / (256 * ADJ_KPT), Nf);
  k_gemv_adj_dd<<<g, 256, sm, s>>>(reinterpret_cast<const float4 *>(A), yh, xh, Nr, Nm);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gemv_adj_cx(const void *A, int fmt, const cdd *yh, cf *xh, int Nf, int Nr, int Nm,
                               cudaStream_t s) {
  const size_t sm = (size_t)Nr * sizeof(AdjRow);
  dim3 g((Nm + 256 * ADJ_KPT - 1) / (256 * ADJ_KPT), Nf);
  if (fmt == FMT_C64) {
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_gemv_adj_cx<FMT_C64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_gemv_adj_cx<FMT_C64><<<g, 256, sm, s>>>(A, yh, xh, Nr, Nm);
  } else if (fmt == FMT_BF16X2) {
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_gemv_adj_cx<FMT_BF16X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_gemv_adj_cx<FMT_BF16X2><<<g, 256, sm, s>>>(A, yh, xh, Nr, Nm);
  } else {
    return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_convert_op(const cdd *src, long src_ld_w, void *dst, int fmt, long dst_ld_w,
                              long n_per_w, int Nf, cudaStream_t s) {
  const long total = (long)Nf * n_per_w;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_convert_op<<<(unsigned)blocks, 256, 0, s>>>(src, src_ld_w, dst, fmt, dst_ld_w, n_per_w, Nf);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tw
