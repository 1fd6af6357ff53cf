// fft_engine.cuh -- batched mixed-radix complex FFT in shared memory.
//
// The FFT-based Toeplitz apply (Sec. "FFT-based Hessian matvecs": embed the
// block Toeplitz matrix in a block circulant one, which the DFT
// block-diagonalises) needs DFTs along time of length 2Nt for many series
// at once, and the Matern prior needs 2D DFTs over the periodic grid.  This
// engine transforms B series of length M held in shared memory with a
// self-sorting (Stockham) sequence of radix-R passes, R in {2,3,4,5,7} with
// specialised butterflies and any other odd R by a direct symmetric DFT.
//
// Pass with radix R, p = product of the earlier radices, S = M/R:
//   for i < S:  k = i mod p,  v_j = in[i + j S] * W_M^(j k M/(p R)),
//               u = DFT_R(v),  out[(i - k) R + k + q p] = u_q.
// After all passes `out` holds DFT_M(in) in natural order.
// W_M^t = exp(-2 pi i t / M) comes from a table; the inverse transform uses
// conj(W) and is unnormalised.
#pragma once
#include "df64.cuh"

namespace tw {

#define TW_FFT_MAX_STAGES 16

struct FftPlan {
  int M;
  int nst;
  int R[TW_FFT_MAX_STAGES];
  // division by p (product of the earlier radices) and by S = M / R of each
  // stage as a multiply-high: q = umulhi(n, mag) then one correction step
  unsigned pmag[TW_FFT_MAX_STAGES], smag[TW_FFT_MAX_STAGES];
};

// n / x and n % x for a divisor x >= 1 with mag = floor(2^32 / x) (x = 1: mag unused)
__device__ __forceinline__ void fdivmod(unsigned n, unsigned x, unsigned mag, unsigned &q, unsigned &r) {
  if (x == 1) { q = n; r = 0; return; }
  q = __umulhi(n, mag);
  r = n - q * x;
  if (r >= x) { ++q; r -= x; }
}

template <class P>
__device__ __forceinline__ typename P::cx ld_cx(const typename P::cx *p);
template <>
__device__ __forceinline__ cdd ld_cx<PolDD>(const cdd *p) {
  float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  cdd r; r.re.hi = v.x; r.re.lo = v.y; r.im.hi = v.z; r.im.lo = v.w; return r;
}
template <>
__device__ __forceinline__ cf ld_cx<PolF>(const cf *p) {
  float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return cf_make(v.x, v.y);
}

template <>
__device__ __forceinline__ cd ld_cx<PolD>(const cd *p) {
  double2 v = __ldg(reinterpret_cast<const double2 *>(p));
  cd r; r.re = v.x; r.im = v.y; return r;
}

// twiddle W_M^t (forward) or its conjugate (inverse)
template <class P, bool INV>
__device__ __forceinline__ typename P::cx twid(const typename P::cx *tab, int t) {
  typename P::cx w = ld_cx<P>(tab + t);
  return INV ? P::conj(w) : w;
}

// Constants of the R-point DFT for odd R: W_R^t = exp(-2 pi i t / R) for
// t = 1..(R-1)/2, read once per pass (the table entry t M / R); W_R^(R-t) is
// their conjugate.  Radix 2 and 4 need none.
template <class P, int R>
struct BflyK {
  typename P::cx w[(R - 1) / 2];
  __device__ __forceinline__ void load(const typename P::cx *tab, int M) {
#pragma unroll
    for (int t = 1; t <= (R - 1) / 2; ++t) w[t - 1] = ld_cx<P>(tab + t * (M / R));
  }
};
template <class P>
struct BflyK<P, 2> { __device__ __forceinline__ void load(const typename P::cx *, int) {} };
template <class P>
struct BflyK<P, 4> { __device__ __forceinline__ void load(const typename P::cx *, int) {} };

// R-point DFT of v (in registers), forward or inverse.
template <class P, bool INV, int R>
struct Bfly;

template <class P, bool INV>
struct Bfly<P, INV, 2> {
  typedef typename P::cx cx;
  static __device__ __forceinline__ void run(cx *v, const BflyK<P, 2> &) {
    cx a = P::add(v[0], v[1]);
    cx b = P::sub(v[0], v[1]);
    v[0] = a; v[1] = b;
  }
};

template <class P, bool INV>
struct Bfly<P, INV, 4> {
  typedef typename P::cx cx;
  static __device__ __forceinline__ void run(cx *v, const BflyK<P, 4> &) {
    cx s02 = P::add(v[0], v[2]), d02 = P::sub(v[0], v[2]);
    cx s13 = P::add(v[1], v[3]), d13 = P::sub(v[1], v[3]);
    // forward: W_4 = -i; inverse: +i
    cx r13 = INV ? P::mul_i(d13) : P::mul_mi(d13);
    v[0] = P::add(s02, s13);
    v[2] = P::sub(s02, s13);
    v[1] = P::add(d02, r13);
    v[3] = P::sub(d02, r13);
  }
};

// odd R: with a_j = v_j + v_{R-j}, b_j = v_j - v_{R-j} (j = 1..h, h = (R-1)/2)
//   u_q     = v_0 + sum_j a_j cos(2 pi j q / R) -/+ i sum_j b_j sin(2 pi j q / R)
//   u_{R-q} = v_0 + sum_j a_j cos(2 pi j q / R) +/- i sum_j b_j sin(2 pi j q / R)
template <class P, bool INV, int R>
struct Bfly {
  typedef typename P::cx cx;
  typedef typename P::re re;
  static __device__ __forceinline__ void run(cx *v, const BflyK<P, R> &K) {
    constexpr int h = (R - 1) / 2;
    cx a[h], b[h];
#pragma unroll
    for (int j = 1; j <= h; ++j) {
      a[j - 1] = P::add(v[j], v[R - j]);
      b[j - 1] = P::sub(v[j], v[R - j]);
    }
    cx u0 = v[0];
#pragma unroll
    for (int j = 0; j < h; ++j) u0 = P::add(u0, a[j]);
#pragma unroll
    for (int q = 1; q <= h; ++q) {
      cx c = v[0];       // v0 + sum a_j cos
      cx s = P::zero();  // sum b_j sin
#pragma unroll
      for (int j = 1; j <= h; ++j) {
        const int t = j * q % R;                      // W_R^t = cos - i sin
        const re cs = P::real(K.w[(t <= h ? t : R - t) - 1]);
        const re si = P::imag(K.w[(t <= h ? t : R - t) - 1]);
        const re sn = t <= h ? si : P::re_neg(si);   // = -sin
        c = P::add(c, P::scale_re(a[j - 1], cs));
        s = P::add(s, P::scale_re(b[j - 1], sn));     // accumulates -sum b sin
      }
      // forward: u_q = c - i * sum b sin = c + i * s ; inverse: c - i * s
      cx is = P::mul_i(s);
      v[q] = INV ? P::sub(c, is) : P::add(c, is);
      v[R - q] = INV ? P::add(c, is) : P::sub(c, is);
    }
    v[0] = u0;
  }
};

// One pass with compile-time radix R.  Buffers: element (b, j) at b*ss + j*es.
template <class P, bool INV, int R>
__device__ __forceinline__ void fft_pass(const typename P::cx *src, typename P::cx *dst,
                                         const typename P::cx *tab, int M, int p, int B,
                                         int es, int ss, bool series_fast, unsigned pmag,
                                         unsigned smag) {
  typedef typename P::cx cx;
  const int S = M / R;
  const int tstride = M / (p * R);
  const int total = S * B;
  const int lgB = __ffs(B) - 1;   // B is a power of two
  BflyK<P, R> K;
  K.load(tab, M);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int b, i;
    if (series_fast) {
      b = idx & (B - 1);
      i = idx >> lgB;
    } else {
      unsigned q, r;
      fdivmod((unsigned)idx, (unsigned)S, smag, q, r);
      i = (int)r;
      b = (int)q;
    }
    unsigned pq, pr;
    fdivmod((unsigned)i, (unsigned)p, pmag, pq, pr);
    const int k = (int)pr;
    cx v[R];
    const cx *sb = src + b * ss;
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = sb[(i + j * S) * es];
    if (k != 0) {
      // j k tstride < (R - 1)(p - 1) M / (p R) < M: no reduction needed
#pragma unroll
      for (int j = 1; j < R; ++j) v[j] = P::mul(v[j], twid<P, INV>(tab, j * k * tstride));
    }
    Bfly<P, INV, R>::run(v, K);
    const int base = (i - k) * R + k;
    cx *db = dst + b * ss;
#pragma unroll
    for (int q = 0; q < R; ++q) db[(base + q * p) * es] = v[q];
  }
}

// Pass with a runtime odd radix R (prime factors above 7).  Step 1, one
// thread per butterfly (each owns its R inputs): twiddle the inputs, replace
// v_j, v_{R-j} (j = 1..h, h = (R-1)/2) in place by a_j = v_j + v_{R-j} and
// b_j = v_j - v_{R-j}, and write u_0 = v_0 + sum a_j.  Step 2, one thread per
// output pair (q, R-q), q = 1..h (the symmetric form of the odd-radix
// butterfly above):  c = v_0 + sum_j a_j cos(2 pi j q/R),
// s = -sum_j b_j sin(2 pi j q/R), u_q = c + i s and u_{R-q} = c - i s
// (forward; swapped for the inverse).  The twiddle index j q mod R advances
// by q per term.  O(R) work per output pair.
template <class P, bool INV>
__device__ void fft_pass_generic(typename P::cx *src, typename P::cx *dst,
                                 const typename P::cx *tab, int M, int p, int R, int B,
                                 int es, int ss, bool series_fast) {
  typedef typename P::cx cx;
  typedef typename P::re re;
  const int S = M / R;
  const int tstride = M / (p * R);
  const int h = (R - 1) / 2;
  const int total = S * B;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int b, i;
    if (series_fast) { b = idx % B; i = idx / B; } else { i = idx % S; b = idx / S; }
    const int k = i % p;
    cx *sb = src + b * ss;
    cx u0 = sb[i * es];
    for (int j = 1; j <= h; ++j) {
      cx vj = sb[(i + j * S) * es], vr = sb[(i + (R - j) * S) * es];
      if (k != 0) {
        // j k tstride < (R - 1)(p - 1) M / (p R) < M: no reduction needed
        vj = P::mul(vj, twid<P, INV>(tab, j * k * tstride));
        vr = P::mul(vr, twid<P, INV>(tab, (R - j) * k * tstride));
      }
      const cx a = P::add(vj, vr);
      sb[(i + j * S) * es] = a;
      sb[(i + (R - j) * S) * es] = P::sub(vj, vr);
      u0 = P::add(u0, a);
    }
    dst[b * ss + ((i - k) * R + k) * es] = u0;
  }
  __syncthreads();
  const int totq = S * h * B;
  for (int idx = threadIdx.x; idx < totq; idx += blockDim.x) {
    int b, i, q;
    if (series_fast) { b = idx % B; const int r = idx / B; i = r % S; q = r / S + 1; }
    else { i = idx % S; const int r = idx / S; b = r % B; q = r / B + 1; }
    const int k = i % p;
    const cx *sb = src + b * ss;
    cx c = sb[i * es];
    cx sn = P::zero();
    int t = 0;
    for (int j = 1; j <= h; ++j) {
      t += q;
      if (t >= R) t -= R;
      const cx w = ld_cx<P>(tab + t * S);              // forward table: cos - i sin
      c = P::add(c, P::scale_re(sb[(i + j * S) * es], P::real(w)));
      sn = P::add(sn, P::scale_re(sb[(i + (R - j) * S) * es], P::imag(w)));
    }
    const cx is = P::mul_i(sn);
    cx *db = dst + b * ss + ((i - k) * R + k) * es;
    db[q * p * es] = INV ? P::sub(c, is) : P::add(c, is);
    db[(R - q) * p * es] = INV ? P::add(c, is) : P::sub(c, is);
  }
}

// Full transform.  Returns the buffer that holds the result (buf0 or buf1).
template <class P, bool INV>
__device__ typename P::cx *fft_run(typename P::cx *buf0, typename P::cx *buf1,
                                   const typename P::cx *tab, const FftPlan &pl, int B,
                                   int es, int ss, bool series_fast) {
  typedef typename P::cx cx;
  cx *src = buf0, *dst = buf1;
  int p = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.R[st];
    const unsigned pm = pl.pmag[st], sm = pl.smag[st];
    switch (R) {
      case 2: fft_pass<P, INV, 2>(src, dst, tab, pl.M, p, B, es, ss, series_fast, pm, sm); break;
      case 3: fft_pass<P, INV, 3>(src, dst, tab, pl.M, p, B, es, ss, series_fast, pm, sm); break;
      case 4: fft_pass<P, INV, 4>(src, dst, tab, pl.M, p, B, es, ss, series_fast, pm, sm); break;
      case 5: fft_pass<P, INV, 5>(src, dst, tab, pl.M, p, B, es, ss, series_fast, pm, sm); break;
      case 7: fft_pass<P, INV, 7>(src, dst, tab, pl.M, p, B, es, ss, series_fast, pm, sm); break;
      default: fft_pass_generic<P, INV>(src, dst, tab, pl.M, p, R, B, es, ss, series_fast); break;
    }
    __syncthreads();
    cx *t = src; src = dst; dst = t;
    p *= R;
  }
  return src;
}

}  // namespace tw
