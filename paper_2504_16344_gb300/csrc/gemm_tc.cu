// gemm_tc.cu -- the batched adjoint product on the 5th-generation tensor cores.
//
// For B right-hand sides the adjoint of the p2o map needs, per frequency w,
//   X^(w) = F^(w)^H Y^(w)          (Nm x Nr) (Nr x B), complex
// (Sec. "FFT-based Hessian matvecs": the block-circulant embedding makes the
// map block diagonal in frequency).  With Ar + i Ai = F^(w) and Y = Yr + i Yi,
//   Xr = Ar^T Yr + Ai^T Yi,   Xi = Ar^T Yi - Ai^T Yr,
// which is one real GEMM D = A' B'^T with K' = 2 Nr:
//   A'[m][2s] = Ar[s][m],  A'[m][2s+1] = Ai[s][m]                  (M = grid points)
//   B'[b][2s] = Yr[s][b],  B'[b][2s+1] = Yi[s][b]       -> D[m][b]      = Xr
//   B'[P+b][2s] = Yi[s][b], B'[P+b][2s+1] = -Yr[s][b]   -> D[m][P+b]    = Xi
// (P = B padded to a multiple of 8, N = 2P <= 256).  The operator is the
// TW_PREC_BF16X2 storage, exactly bf16 hi + bf16 lo (Ah + Al); B' (FP32) is
// split into three bf16 terms Bh + Bm + Bl (a 2^-27 representation: a two-term
// split's 2^-18 error showed in m), and D accumulates
// Ah (Bh + Bm + Bl) + Al (Bh + Bm) in FP32 -- five MMAs per 16-wide k step;
// the dropped Al Bl is below 2^-26 of the product.
//
// Layout: the operator is re-stored once (tw_reserve_batch) as the shared-
// memory image the MMA reads -- per (frequency, 128-point tile, 64-wide K'
// atom, hi/lo) a 128 x 64 bf16 tile, K-major, 128-byte swizzle (16-byte
// chunk j of row r at chunk j ^ (r mod 8)) -- so one 16 KB bulk copy (TMA
// engine, cp.async.bulk) moves a ready operand.  B' tiles are written in the
// same form per frequency by k_btc_build.
//
// One CTA (4 warps) per (128-point tile, frequency, slice of up to 128
// right-hand sides): thread 0 issues the bulk copies (mbarrier with
// transaction count) and the MMAs (tcgen05.mma, one elected thread, D in
// TMEM); completion is signalled through tcgen05.commit on an mbarrier; each
// warp then reads its 32 TMEM lanes (tcgen05.ld) and writes complex64 X.
// Every wait is bounded; on expiry the kernel records TW_ERR_TIMEOUT, waits
// (bounded) for its own copies and MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/tw.h"
#include "kernels.h"

namespace tw {

namespace {

constexpr int TM = 128;                 // MMA M: grid points per tile
constexpr int KA = 64;                  // K' per 128-byte swizzle atom
constexpr int ATOM_A = TM * KA * 2;     // bytes of one operator tile (16 KB)
constexpr unsigned SPIN_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, j) in a K-major 128-byte-swizzled tile of 64 bf16 per row
__host__ __device__ __forceinline__ uint32_t swz(int row, int j) {
  return (uint32_t)row * 128u + ((uint32_t)((j >> 3) ^ (row & 7)) << 4) + (uint32_t)(j & 7) * 2u;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); the leading-dimension offset is unused for this
// layout; bits 46-47 = 1 (tcgen05 descriptor version), bits 61-63 = 2 (128B swizzle)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase with this parity has completed; false after the spin limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity) {
  for (unsigned it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.b32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, unsigned bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\t"
               "setp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
               ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(bar) : "memory");
}

// ------------------------------------------------------------ operand builds
// operator: tiles [w][mt][ka][hl][128][64] from the bf16x2 storage [w][s][m]
// (uint2 per complex entry: word = hi | lo << 16 for re (x) and im (y))
__global__ void k_optc_build(const uint2 *__restrict__ op, uint8_t *__restrict__ tc, int Nr, int Nm,
                             int nmt, int nka) {
  const int w = blockIdx.z, mt = blockIdx.y, ka = blockIdx.x;
  uint8_t *base = tc + ((((size_t)w * nmt + mt) * nka + ka) * 2) * ATOM_A;
  for (int e = threadIdx.x; e < TM * KA; e += blockDim.x) {
    const int r = e >> 6, j = e & 63;
    const int m = mt * TM + r, kk = ka * KA + j, s = kk >> 1;
    unsigned short hi = 0, lo = 0;
    if (m < Nm && s < Nr) {
      const uint2 v = op[((size_t)w * Nr + s) * Nm + m];
      const unsigned word = (kk & 1) ? v.y : v.x;
      hi = (unsigned short)(word & 0xffffu);
      lo = (unsigned short)(word >> 16);
    }
    const uint32_t off = swz(r, j);
    *reinterpret_cast<unsigned short *>(base + off) = hi;
    *reinterpret_cast<unsigned short *>(base + ATOM_A + off) = lo;
  }
}

// B' tiles of one slice: [w][ka][term][N][64] (term hi, mid, lo), rows n < P
// real-part columns, n >= P imaginary
__global__ void k_btc_build(const cf *__restrict__ Y, long y_bstride, uint8_t *__restrict__ btc,
                            int Nf, int Nr, int B, int P, int nka) {
  const int w = blockIdx.y, ka = blockIdx.x;
  const int N = 2 * P;
  const size_t tile = (size_t)N * 128;
  uint8_t *base = btc + (((size_t)w * nka + ka) * 3) * tile;
  for (int e = threadIdx.x; e < N * KA; e += blockDim.x) {
    const int n = e >> 6, j = e & 63;
    const int kk = ka * KA + j, s = kk >> 1, c = kk & 1;
    const int part = n >= P, b = n - part * P;
    float v = 0.f;
    if (b < B && s < Nr) {
      const cf y = Y[(size_t)b * y_bstride + (size_t)w * Nr + s];
      v = part == 0 ? (c == 0 ? y.re : y.im) : (c == 0 ? y.im : -y.re);
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);            // exact in FP32
    const __nv_bfloat16 mdl = __float2bfloat16_rn(r1);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(mdl));
    const uint32_t off = swz(n, j);
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = h;
    *reinterpret_cast<__nv_bfloat16 *>(base + tile + off) = mdl;
    *reinterpret_cast<__nv_bfloat16 *>(base + 2 * tile + off) = l;
  }
}

// ------------------------------------------------------------------ the GEMM
__global__ void __launch_bounds__(128)
k_gemm_adj_tc(const uint8_t *__restrict__ Atc, const uint8_t *__restrict__ Btc, cf *__restrict__ X,
              long x_bstride, int b0, int Nm, int nmt, int nka, int ksteps, int B, int P,
              unsigned tmem_cols, int *err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, w = blockIdx.y;
  const int N = 2 * P;
  const uint32_t btile = (uint32_t)N * 128u;
  // 1024-byte aligned operand area: A hi | A lo | B hi | B mid | B lo
  const uint32_t sbase = (su32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sA = sbase, sB = sbase + 2 * ATOM_A;
  const uint32_t bar_full = su32(&bars[0]), bar_mma = su32(&bars[1]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(su32(&tmem_slot)), "r"(tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    fail = 0;
    mbar_init(bar_full, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_bf16(TM, N);
  unsigned parity = 0;
  if (tid == 0) {
    const uint8_t *Ablk = Atc + (((size_t)w * nmt + mt) * nka) * 2 * ATOM_A;
    const uint8_t *Bblk = Btc + ((size_t)w * nka) * 3 * btile;
    bool ok = true;
    for (int ka = 0; ka < nka && ok; ++ka) {
      mbar_expect_tx(bar_full, 2 * ATOM_A + 3 * btile);
      bulk_g2s(sA, Ablk + (size_t)ka * 2 * ATOM_A, 2 * ATOM_A, bar_full);
      bulk_g2s(sB, Bblk + (size_t)ka * 3 * btile, 3 * btile, bar_full);
      ok = mbar_wait(bar_full, parity);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int ks = 0; ks < KA / 16; ++ks) {
        const int kk = ka * (KA / 16) + ks;
        if (kk >= ksteps) break;
        const uint64_t a_hi = sdesc(sA + ks * 32), a_lo = sdesc(sA + ATOM_A + ks * 32);
        const uint64_t b_hi = sdesc(sB + ks * 32), b_md = sdesc(sB + btile + ks * 32);
        const uint64_t b_lo = sdesc(sB + 2 * btile + ks * 32);
        mma_bf16(tmem, a_hi, b_hi, idesc, kk > 0 ? 1u : 0u);
        mma_bf16(tmem, a_hi, b_md, idesc, 1u);
        mma_bf16(tmem, a_hi, b_lo, idesc, 1u);
        mma_bf16(tmem, a_lo, b_hi, idesc, 1u);
        mma_bf16(tmem, a_lo, b_md, idesc, 1u);
      }
      mma_commit(bar_mma);                     // MMAs done -> operands reusable, D final
      ok = mbar_wait(bar_mma, parity);
      parity ^= 1u;
    }
    if (!ok) {
      fail = 1;
      if (atomicCAS(err, 0, TW_ERR_TIMEOUT) == 0) err[1] = 20;
      // let copies and MMAs already issued drain (bounded) before TMEM is freed
      mma_commit(bar_mma);
      mbar_wait(bar_mma, parity);
      mbar_wait(bar_full, parity);
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!fail) {
    // warp q reads TMEM lanes 32q..32q+31: row m = mt*128 + 32q + lane
    const int m = mt * TM + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < P; c0 += 16) {
      uint32_t re[16], im[16];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]),
                     "=r"(re[6]), "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]),
                     "=r"(re[12]), "=r"(re[13]), "=r"(re[14]), "=r"(re[15])
                   : "r"(trow + (uint32_t)c0));
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]),
                     "=r"(im[6]), "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]),
                     "=r"(im[12]), "=r"(im[13]), "=r"(im[14]), "=r"(im[15])
                   : "r"(trow + (uint32_t)(P + c0)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < Nm) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int b = c0 + j;
          if (b < B)
            X[(size_t)(b0 + b) * x_bstride + (size_t)w * Nm + m] =
                cf_make(__uint_as_float(re[j]), __uint_as_float(im[j]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
}

}  // namespace

// ------------------------------------------------------------------ host side
int gemm_tc_nka(int Nr) { return (2 * Nr + KA - 1) / KA; }
int gemm_tc_nmt(int Nm) { return (Nm + TM - 1) / TM; }
size_t gemm_tc_op_bytes(int Nf, int Nr, int Nm) {
  return (size_t)Nf * gemm_tc_nmt(Nm) * gemm_tc_nka(Nr) * 2 * ATOM_A;
}
// B' workspace for slices of up to 128 right-hand sides
size_t gemm_tc_b_bytes(int Nf, int Nr) { return (size_t)Nf * gemm_tc_nka(Nr) * 3 * 256 * 128; }

cudaError_t launch_optc_build(const void *op_bf16x2, void *tc, int Nf, int Nr, int Nm,
                              cudaStream_t s) {
  dim3 grid(gemm_tc_nka(Nr), gemm_tc_nmt(Nm), Nf);
  k_optc_build<<<grid, 256, 0, s>>>(reinterpret_cast<const uint2 *>(op_bf16x2),
                                    reinterpret_cast<uint8_t *>(tc), Nr, Nm, gemm_tc_nmt(Nm),
                                    gemm_tc_nka(Nr));
  count_launches(1);
  return cudaGetLastError();
}

// X[b][w][k] = sum_s conj(F^[w][s][k]) Y[b][w][s], b < B (any B: slices of 128)
cudaError_t launch_gemm_adj_tc(const void *op_tc, const cf *Y, long y_bstride, cf *X,
                               long x_bstride, int Nf, int Nr, int Nm, int B, void *btc, int *err,
                               cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int nka = gemm_tc_nka(Nr), nmt = gemm_tc_nmt(Nm), ksteps = (2 * Nr + 15) / 16;
  for (int b0 = 0; b0 < B; b0 += 128) {
    const int nb = B - b0 < 128 ? B - b0 : 128;
    const int P = (nb + 7) / 8 * 8;
    const int N = 2 * P;
    unsigned cols = 32;
    while ((int)cols < N) cols <<= 1;
    k_btc_build<<<dim3(nka, Nf), 256, 0, s>>>(Y + (size_t)b0 * y_bstride, y_bstride,
                                              reinterpret_cast<uint8_t *>(btc), Nf, Nr, nb, P, nka);
    count_launches(1);
    const size_t sm = 1024 + 2 * (size_t)ATOM_A + 3 * (size_t)N * 128;
    cudaFuncSetAttribute(k_gemm_adj_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_gemm_adj_tc<<<dim3(nmt, Nf), 128, sm, s>>>(reinterpret_cast<const uint8_t *>(op_tc),
                                                 reinterpret_cast<const uint8_t *>(btc), X, x_bstride,
                                                 b0, Nm, nmt, nka, ksteps, nb, P, cols, err);
    count_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace tw
