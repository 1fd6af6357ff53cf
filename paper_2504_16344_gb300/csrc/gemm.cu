// gemm.cu -- the per-frequency products for a batch of right-hand sides.
//
// With B right-hand sides the block-diagonal-in-frequency form of the
// Toeplitz maps (Sec. "FFT-based Hessian matvecs") turns each frequency's
// matrix-vector product into a matrix-matrix product:
//   adjoint  X^(w) = F^(w)^H Y^(w)      (Nm x Nr) (Nr x B)
//   forward  Y^(w) = F^(w)   X^(w)      (Nr x Nm) (Nm x B)
// The operator is read once per CTA column slice instead of once per
// right-hand side, so the cost moves from HBM to the arithmetic units.
//
// Batched arrays are RHS-major: entry b of Y is at Y + b * y_bstride and
// holds [Nf][Nr] complex values (X: [Nf][Nm]).
//
//  * adjoint: a CTA owns 128 grid points of one frequency and a slice of
//    right-hand sides; its slice of Y^(w) sits in shared memory, each warp
//    keeps 4 right-hand sides x 4 grid points of accumulators and walks the
//    Nr rows (no cross-thread reduction).
//  * forward: a CTA owns a range of grid points of one frequency and 32
//    right-hand sides (lane = right-hand side); each warp keeps RPW rows of
//    accumulators, reads F^(w) entries once (broadcast to the warp) and the
//    X^(w) tile from shared memory.  The per-range partial sums are added by
//    a second kernel in a fixed order.
//
// FP64-class path: float-pair operands, exact products, renormalised
// running sums (as the single-vector kernels).  Reduced-precision paths:
// complex64 or bf16 hi+lo operator, the forward product in FP32 FMA (their
// adjoint runs on the tensor cores: gemm_sl.cu).
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace tw {

namespace {

constexpr int GA_K = 128;      // grid points per CTA (adjoint)
constexpr int GF_K = 128;      // grid points per shared tile (forward)
constexpr int GF_TILES = 32;   // tiles per CTA: a CTA sums 4096 grid points

__device__ __forceinline__ float bf16lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }

// ------------------------------------------------------------ adjoint, df64
// grid (ceil(Nm/128), Nf, ceil(B/(8 RW))); 8 warps x RW right-hand sides each
// (RW = 4, 2 or 1 after the batch size, so small batches leave no warp idle)
template <int RW>
__global__ void __launch_bounds__(256, 2)
k_gemm_adj_dd(const float4 *__restrict__ A, const cdd *__restrict__ Y, long y_bstride,
              cdd *__restrict__ X, long x_bstride, int Nr, int Nm, int B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CB = 8 * RW;                      // right-hand sides per CTA
  cdd *sy = reinterpret_cast<cdd *>(smem_raw);   // [CB][Nr]
  const int w = blockIdx.y;
  const int b0 = blockIdx.z * CB;
  const int nb = min(CB, B - b0);
  for (int idx = threadIdx.x; idx < CB * Nr; idx += blockDim.x) {
    const int bl = idx / Nr, sr = idx % Nr;
    sy[idx] = bl < nb ? ld_cdd(Y + (size_t)(b0 + bl) * y_bstride + (size_t)w * Nr + sr) : cdd_zero();
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int k0 = blockIdx.x * GA_K + lane;
  const float4 *Aw = A + (size_t)w * Nr * Nm;
  dacc re[RW][4], im[RW][4];   // [rhs][point]
  bool ok[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) ok[j] = k0 + 32 * j < Nm;
#pragma unroll
  for (int i = 0; i < RW; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { re[i][j] = dacc_zero(); im[i][j] = dacc_zero(); }
  float4 cur[4], nxt[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) cur[j] = ok[j] ? __ldg(Aw + k0 + 32 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
  const cdd *syg = sy + (grp * RW) * Nr;
  for (int s = 0; s < Nr; ++s) {
    if (s + 1 < Nr) {
      const float4 *row = Aw + (size_t)(s + 1) * Nm + k0;
#pragma unroll
      for (int j = 0; j < 4; ++j) nxt[j] = ok[j] ? __ldg(row + 32 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < RW; ++i) {
      const cdd y = syg[i * Nr + s];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        dd ar, ai;
        ar.hi = cur[j].x; ar.lo = cur[j].y; ai.hi = cur[j].z; ai.lo = cur[j].w;
        // conj(a) y = (ar yr + ai yi) + i (ar yi - ai yr)
        dacc_mac(re[i][j], ar, y.re);
        dacc_mac(re[i][j], ai, y.im);
        dacc_mac(im[i][j], ar, y.im);
        dacc_mac(im[i][j], dd_neg(ai), y.re);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) cur[j] = nxt[j];
  }
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    const int bl = grp * RW + i;
    if (bl >= nb) continue;
    cdd *xo = X + (size_t)(b0 + bl) * x_bstride + (size_t)w * Nm;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!ok[j]) continue;
      cdd r;
      r.re = dacc_get(re[i][j]);
      r.im = dacc_get(im[i][j]);
      st_cdd(xo + k0 + 32 * j, r);
    }
  }
}

// ----------------------------------------- adjoint, FP32 operator, pair data
// ------------------------------------------------------------ forward
// grid (nchunk, Nf, ceil(B/32)); a CTA sums 4096 grid points of one
// frequency for 32 right-hand sides (lane = right-hand side) and all Nr rows
// (warp w owns rows w, w+8, ..., RPW of them per pass).  Each GK-wide k
// tile stages X^ [32][GK] and the operator rows [Nr][GK] in shared memory;
// the inner loop reads the operator entry as a warp broadcast and X^ per
// lane, both from shared memory.  Partial sums per chunk go to
// part[b][w][chunk][r].
template <class CX> struct FwdT;
template <> struct FwdT<cdd> {
  typedef dacc acc;
  static __device__ __forceinline__ void zero(acc &re, acc &im) { re = dacc_zero(); im = dacc_zero(); }
  // (re, im) += a x
  static __device__ __forceinline__ void mac(acc &re, acc &im, const cdd &a, const cdd &x) {
    dacc_mac(re, a.re, x.re);
    dacc_mac(re, dd_neg(a.im), x.im);
    dacc_mac(im, a.re, x.im);
    dacc_mac(im, a.im, x.re);
  }
  static __device__ __forceinline__ cdd get(const acc &re, const acc &im) {
    cdd r; r.re = dacc_get(re); r.im = dacc_get(im); return r;
  }
  static __device__ __forceinline__ cdd zx() { return cdd_zero(); }
  // add the partner lane's partial sum (lane ^ m)
  static __device__ __forceinline__ void combine(acc &a, int m) {
    dd o;
    o.hi = __shfl_xor_sync(0xffffffffu, a.s, m);
    o.lo = __shfl_xor_sync(0xffffffffu, a.t, m);
    dacc_add(a, o);
  }
};
template <> struct FwdT<cf> {
  typedef float acc;
  static __device__ __forceinline__ void zero(acc &re, acc &im) { re = 0.f; im = 0.f; }
  static __device__ __forceinline__ void mac(acc &re, acc &im, const cf &a, const cf &x) {
    re = fmaf(a.re, x.re, fmaf(-a.im, x.im, re));
    im = fmaf(a.re, x.im, fmaf(a.im, x.re, im));
  }
  static __device__ __forceinline__ cf get(const acc &re, const acc &im) { return cf_make(re, im); }
  static __device__ __forceinline__ cf zx() { return cf_zero(); }
  static __device__ __forceinline__ void combine(acc &a, int m) {
    a += __shfl_xor_sync(0xffffffffu, a, m);
  }
};


// one element copied to shared memory asynchronously (zero-filled if !ok; the
// source is then only a valid address, nothing is read from it)
template <class CX>
__device__ __forceinline__ void cp_async_el(CX *dst, const CX *src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(CX) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}

// LPB lanes per right-hand side: 1 (32 right-hand sides per CTA) or 2 (16;
// the two lanes of a right-hand side take alternate k and add their sums
// at the end), so batches of up to 16 leave no lane idle.  The caller fixes
// LPB per context (from the reserved batch), so a right-hand side's sum
// order never depends on what shares its batch.
template <class CX, int RPW, int GK, int FMT, int LPB>
__global__ void __launch_bounds__(256, 2)
k_gemm_fwd(const void *__restrict__ A, const CX *__restrict__ X, long x_bstride,
           CX *__restrict__ part, int nchunk, int Nr, int Nm, int B) {
  typedef FwdT<CX> T;
  constexpr int CB = 32 / LPB;                        // right-hand sides per CTA
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CX *sx = reinterpret_cast<CX *>(smem_raw);          // [CB][GK + 1]
  CX *sa = sx + CB * (GK + 1);                        // [Nr][GK]
  const int w = blockIdx.y, chunk = blockIdx.x;
  const int b0 = blockIdx.z * CB;
  const int nb = min(CB, B - b0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bl_l = lane % CB, half = lane / CB;       // right-hand side, k phase
  const int kbeg = chunk * GF_K * GF_TILES;
  const int kend = min(Nm, kbeg + GF_K * GF_TILES);
  const size_t base = (size_t)w * Nr * Nm;
  const int npass = (Nr + 8 * RPW - 1) / (8 * RPW);
  for (int pass = 0; pass < npass; ++pass) {
    const int r0 = pass * 8 * RPW;
    const int nrp = min(8 * RPW, Nr - r0);           // rows staged this pass
    typename T::acc re[RPW], im[RPW];
#pragma unroll
    for (int i = 0; i < RPW; ++i) T::zero(re[i], im[i]);
    for (int kt = kbeg; kt < kend; kt += GK) {
      const int nk = min(GK, kend - kt);
      __syncthreads();   // previous tile consumed
      {
        // every load of the tile in flight at once (cp.async, zeros past the
        // edges); bf16 hi+lo words are copied as they are stored (8 bytes,
        // the size of the complex64 slot) and converted in place below
        static_assert(sizeof(CX) == 16 || FMT != FMT_DD, "float-pair tile");
        const CX *Ac = reinterpret_cast<const CX *>(A);
        for (int idx = threadIdx.x; idx < CB * GK; idx += blockDim.x) {
          const int bl = idx / GK, kk = idx % GK;
          const bool ok = bl < nb && kk < nk;
          cp_async_el(sx + bl * (GK + 1) + kk,
                      ok ? X + (size_t)(b0 + bl) * x_bstride + (size_t)w * Nm + kt + kk : X, ok);
        }
        for (int idx = threadIdx.x; idx < nrp * GK; idx += blockDim.x) {
          const int rl = idx / GK, kk = idx % GK;
          const bool ok = kk < nk;
          cp_async_el(sa + rl * GK + kk, ok ? Ac + base + (size_t)(r0 + rl) * Nm + kt + kk : Ac, ok);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
        if constexpr (FMT == FMT_BF16X2) {
          // a thread converts the words it copied itself (visible to it after the wait)
          for (int idx = threadIdx.x; idx < nrp * GK; idx += blockDim.x) {
            CX *e = sa + (idx / GK) * GK + idx % GK;
            const uint2 v = *reinterpret_cast<const uint2 *>(e);
            *e = cf_make(bf16lo(v.x) + bf16hi(v.x), bf16lo(v.y) + bf16hi(v.y));
          }
        }
      }
      __syncthreads();
      const CX *xs = sx + bl_l * (GK + 1);
      if constexpr (std::is_same<CX, cf>::value) {
        // FP32: a fresh sum per tile, added to the running total, so rounding
        // grows with GK + the tile count rather than the chunk length
        float tre[RPW], tim[RPW];
#pragma unroll
        for (int i = 0; i < RPW; ++i) { tre[i] = 0.f; tim[i] = 0.f; }
#pragma unroll 4
        for (int kk = half; kk < nk; kk += LPB) {
          const CX x = xs[kk];
#pragma unroll
          for (int i = 0; i < RPW; ++i) {
            const int rl = warp * RPW + i;
            if (rl < nrp) T::mac(tre[i], tim[i], sa[rl * GK + kk], x);
          }
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) { re[i] += tre[i]; im[i] += tim[i]; }
      } else {
#pragma unroll 4
        for (int kk = half; kk < nk; kk += LPB) {
          const CX x = xs[kk];
#pragma unroll
          for (int i = 0; i < RPW; ++i) {
            const int rl = warp * RPW + i;
            if (rl < nrp) T::mac(re[i], im[i], sa[rl * GK + kk], x);
          }
        }
      }
    }
    if (LPB == 2) {
#pragma unroll
      for (int i = 0; i < RPW; ++i) { T::combine(re[i], 16); T::combine(im[i], 16); }
    }
    if (half == 0 && bl_l < nb) {
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        const int rl = warp * RPW + i;
        if (rl >= nrp) continue;
        part[(((size_t)(b0 + bl_l) * gridDim.y + w) * nchunk + chunk) * Nr + r0 + rl] = T::get(re[i], im[i]);
      }
    }
  }
}

// out[b][w][r] = sum over chunks (ascending) of part[b][w][chunk][r]
__global__ void k_gemm_fwd_reduce_dd(const cdd *__restrict__ part, cdd *__restrict__ Yo,
                                     long y_bstride, int nchunk, int Nf, int Nr, int B) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)B * Nf * Nr;
  if (i >= total) return;
  const int r = (int)(i % Nr);
  const long bw = i / Nr;
  const int w = (int)(bw % Nf), b = (int)(bw / Nf);
  const cdd *p = part + (size_t)bw * nchunk * Nr + r;
  cdd acc = cdd_zero();
  for (int c = 0; c < nchunk; ++c) acc = cdd_add(acc, ld_cdd(p + (size_t)c * Nr));
  st_cdd(Yo + (size_t)b * y_bstride + (size_t)w * Nr + r, acc);
}
__global__ void k_gemm_fwd_reduce_f(const cf *__restrict__ part, cf *__restrict__ Yo,
                                    long y_bstride, int nchunk, int Nf, int Nr, int B) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)B * Nf * Nr;
  if (i >= total) return;
  const int r = (int)(i % Nr);
  const long bw = i / Nr;
  const int w = (int)(bw % Nf), b = (int)(bw / Nf);
  const cf *p = part + (size_t)bw * nchunk * Nr + r;
  cf acc = cf_zero();
  for (int c = 0; c < nchunk; ++c) acc = cf_add(acc, p[(size_t)c * Nr]);
  Yo[(size_t)b * y_bstride + (size_t)w * Nr + r] = acc;
}

template <class KER>
void ensure_smem_g(KER k, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int gemm_fwd_nchunk(int Nm) { return (Nm + GF_K * GF_TILES - 1) / (GF_K * GF_TILES); }

// right-hand sides per warp of the adjoint products: 4 (32 per CTA) for
// large batches, fewer for small ones so that no warp computes empty columns
static int adj_rw(int B) { return B > 16 ? 4 : (B > 8 ? 2 : 1); }

template <int RW>
static void adj_dd_run(const void *A, const cdd *Y, long y_bstride, cdd *X, long x_bstride, int Nf,
                       int Nr, int Nm, int B, cudaStream_t s) {
  const size_t sm = (size_t)8 * RW * Nr * sizeof(cdd);
  ensure_smem_g(k_gemm_adj_dd<RW>, sm);
  dim3 grid((Nm + GA_K - 1) / GA_K, Nf, (B + 8 * RW - 1) / (8 * RW));
  k_gemm_adj_dd<RW><<<grid, 256, sm, s>>>(reinterpret_cast<const float4 *>(A), Y, y_bstride, X,
                                          x_bstride, Nr, Nm, B);
}

cudaError_t launch_gemm_adj_dd(const void *A, const cdd *Y, long y_bstride, cdd *X, long x_bstride,
                               int Nf, int Nr, int Nm, int B, cudaStream_t s, int rw) {
  if (B <= 0) return cudaSuccess;
  if (rw != 0 && rw != 1 && rw != 2 && rw != 4) return cudaErrorInvalidValue;
  switch (rw ? rw : adj_rw(B)) {
    case 4: adj_dd_run<4>(A, Y, y_bstride, X, x_bstride, Nf, Nr, Nm, B, s); break;
    case 2: adj_dd_run<2>(A, Y, y_bstride, X, x_bstride, Nf, Nr, Nm, B, s); break;
    default: adj_dd_run<1>(A, Y, y_bstride, X, x_bstride, Nf, Nr, Nm, B, s); break;
  }
  count_launches(1);
  return cudaGetLastError();
}

// rows per warp: one pass covers up to 8*RPW rows
template <class CX, int RPW, int GK, int FMT, int LPB>
static cudaError_t gemm_fwd_run(const void *A, const CX *X, long x_bstride, CX *part, int Nf, int Nr,
                                int Nm, int B, cudaStream_t s) {
  const int nchunk = gemm_fwd_nchunk(Nm);
  const int rows = std::min(Nr, 8 * RPW);
  const size_t sm = (size_t)((32 / LPB) * (GK + 1) + rows * GK) * sizeof(CX);
  ensure_smem_g(k_gemm_fwd<CX, RPW, GK, FMT, LPB>, sm);
  dim3 grid(nchunk, Nf, (B + 32 / LPB - 1) / (32 / LPB));
  k_gemm_fwd<CX, RPW, GK, FMT, LPB><<<grid, 256, sm, s>>>(A, X, x_bstride, part, nchunk, Nr, Nm, B);
  count_launches(1);
  return cudaGetLastError();
}

template <class CX, int GK, int FMT>
static cudaError_t gemm_fwd_pick(const void *A, const CX *X, long x_bstride, CX *part, int Nf, int Nr,
                                 int Nm, int B, int lpb, cudaStream_t s) {
  // rows per warp: the smallest of 3, 7, 13 that spreads Nr rows over the 8
  // warps in one pass (13 and several passes beyond 104 rows)
  if (lpb == 2) {
    if (Nr <= 24) return gemm_fwd_run<CX, 3, GK, FMT, 2>(A, X, x_bstride, part, Nf, Nr, Nm, B, s);
    if (Nr <= 56) return gemm_fwd_run<CX, 7, GK, FMT, 2>(A, X, x_bstride, part, Nf, Nr, Nm, B, s);
    return gemm_fwd_run<CX, 13, GK, FMT, 2>(A, X, x_bstride, part, Nf, Nr, Nm, B, s);
  }
  if (Nr <= 24) return gemm_fwd_run<CX, 3, GK, FMT, 1>(A, X, x_bstride, part, Nf, Nr, Nm, B, s);
  if (Nr <= 56) return gemm_fwd_run<CX, 7, GK, FMT, 1>(A, X, x_bstride, part, Nf, Nr, Nm, B, s);
  return gemm_fwd_run<CX, 13, GK, FMT, 1>(A, X, x_bstride, part, Nf, Nr, Nm, B, s);
}

cudaError_t launch_gemm_fwd_dd(const void *A, const cdd *X, long x_bstride, cdd *part, cdd *Yo,
                               long y_bstride, int Nf, int Nr, int Nm, int B, cudaStream_t s,
                               int lpb) {
  if (B <= 0) return cudaSuccess;
  cudaError_t e = gemm_fwd_pick<cdd, 32, FMT_DD>(A, X, x_bstride, part, Nf, Nr, Nm, B, lpb, s);
  if (e != cudaSuccess) return e;
  const int nchunk = gemm_fwd_nchunk(Nm);
  const long total = (long)B * Nf * Nr;
  k_gemm_fwd_reduce_dd<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, Yo, y_bstride, nchunk,
                                                                      Nf, Nr, B);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gemm_fwd_f(const void *A, int fmt, const cf *X, long x_bstride, cf *part,
                              cf *Yo, long y_bstride, int Nf, int Nr, int Nm, int B,
                              cudaStream_t s, int lpb) {
  if (B <= 0) return cudaSuccess;
  cudaError_t e;
  if (fmt == FMT_C64)
    e = gemm_fwd_pick<cf, 64, FMT_C64>(A, X, x_bstride, part, Nf, Nr, Nm, B, lpb, s);
  else
    e = gemm_fwd_pick<cf, 64, FMT_BF16X2>(A, X, x_bstride, part, Nf, Nr, Nm, B, lpb, s);
  if (e != cudaSuccess) return e;
  const int nchunk = gemm_fwd_nchunk(Nm);
  const long total = (long)B * Nf * Nr;
  k_gemm_fwd_reduce_f<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, Yo, y_bstride, nchunk,
                                                                     Nf, Nr, B);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tw
