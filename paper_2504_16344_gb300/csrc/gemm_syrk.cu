// gemm_syrk.cu -- K's block products P = G G^T on the 5th-generation tensor
// cores, with G cut into exact fixed-point bf16 slices.
//
// Phase 2 forms K = sigma^2 I + F Gamma_pr F^T (Sec. "Real-time Bayesian
// inference and prediction framework"); with G = Phi C^{1/2} the block
// products are P = G G^T, a symmetric rank-Nm product over the grid, followed
// by prefix sums along the block diagonals (dense.cu).  K is factored in FP64
// and its conditioning amplifies rounding in these long sums, so P is needed
// to FP64 level.
//
// Slices.  Row i of G gets a power-of-two exponent e_i with |G_ik| < 2^e_i for
// every k, and each entry is written in fixed point as seven 8-bit integer
// slices (round to nearest at each step):
//   G_ik = 2^(e_i - 7) (s0 + s1 / 2^8 + ... + s6 / 2^48),  |s_p| <= 128,
// 55 bits below the row maximum (the double-float G has 48 bits of its own).
// Slice p is stored pre-scaled, s_p 2^-8p, exact in bf16.  The product of
// slices p and q is a multiple of 2^-8(p+q) of magnitude <= 2^14 2^-8(p+q);
// level L = p + q collects the L + 1 pairs of that scale, and pairs with
// L <= 6 are formed (28 MMAs per 16-wide k step; the dropped levels are
// below 2^-56 of a term).
//
// Exact accumulation.  The tensor cores accumulate in FP32 and truncate.  A
// level's sum over a chunk of 128 k is a multiple of 2^-8L below
// (L+1) 128 2^14 2^-8L <= 5 2^21 2^-8L for L <= 4, an integer count below
// 2^24: levels 0 .. 4 each accumulate EXACTLY in their own TMEM accumulator.
// Levels 5 and 6 share a sixth (2^-40 below a term, where the truncation of
// its ~100 accumulation steps stays near 2^-56 of the terms).  After each
// chunk the epilogue reads the six accumulators, scales each D_L by 2^8L to
// an integer D_L' and forms the exact
//   X = ((((D0' 2^8 + D1') 2^8 + D2') 2^8 + D3') 2^8 + D4') = (D0 + .. + D4) 2^32,
// adds it to an int64 total (exact) and D56 to an FP32 total.  At the end of
// a panel of k the tile adds 2^(e_i + e_j - 14) (T 2^-32 + F) to K in FP64:
// one rounding per panel.
//
// Kernel: persistent, one CTA per SM, over a host-ordered list of (128-row,
// 32-column) tiles of the lower triangle (groups of 8 row tiles, column tile
// outer, so the CTAs running together share their slice tiles in L2).  One
// thread issues the bulk copies of a k atom's slices (A: 7 x 128 rows, B: 7 x
// 32 rows of the same sliced panel) into a 3-stage ring; one thread issues
// the MMAs (six accumulators of 32 columns, double-buffered per chunk); four
// warps drain TMEM (tcgen05.ld), one row each.  Every wait is bounded: on
// expiry the kernel records TW_ERR_TIMEOUT, lets its copies and MMAs drain
// (bounded), frees TMEM and returns.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/tw.h"
#include "dense_api.h"
#include "kernels.h"

namespace tw {

namespace {

constexpr int SK_TM = 128;                   // MMA M: rows of a tile
constexpr int SK_TN = 32;                    // MMA N: columns of a tile
constexpr int SK_KA = 32;                    // k per atom (two 16-wide MMA steps)
constexpr int SK_NSL = 7;                    // slices per entry
constexpr int SK_NACC = 6;                   // accumulators: levels 0 .. 4, and 5..6
constexpr int SK_CHUNK = 4;                  // atoms per exact chunk (128 k)
constexpr int SK_A_SLICE = SK_TM * SK_KA * 2;     // 8 KB
constexpr int SK_B_SLICE = SK_TN * SK_KA * 2;     // 2 KB
constexpr int SK_A_STAGE = SK_NSL * SK_A_SLICE;   // 56 KB
constexpr int SK_B_STAGE = SK_NSL * SK_B_SLICE;   // 14 KB
constexpr int SK_STAGE = SK_A_STAGE + SK_B_STAGE; // 70 KB
constexpr int SK_S = 3;                      // ring stages
constexpr int SK_NEPI = 128;                 // epilogue threads
constexpr int SK_NTHR = 64 + SK_NEPI;        // copy warp, MMA warp, 4 epilogue warps
constexpr unsigned long long SK_WAIT_NS = 4000000000ull;   // bound of every wait (4 s)
constexpr int SK_EXP_MIN = -100, SK_EXP_MAX = 120;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__host__ __device__ __forceinline__ uint32_t swz64(int r, int q) {
  return (uint32_t)r * 64u + ((uint32_t)(q ^ ((r >> 1) & 3)) << 4);
}
// K-major, 64-byte swizzle, 8-row groups 512 bytes apart (descriptor version 1)
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// kind::f16: D F32, A and B BF16, both K-major
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, unsigned parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\t"
               "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.b32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// true once the phase of this parity has completed; false after SK_WAIT_NS
// or once another role of the CTA has failed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity, volatile int *fail) {
  unsigned long long t0 = 0;
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*fail) return false;
      const unsigned long long t = gtime();
      if (t0 == 0) t0 = t;
      else if (t - t0 > SK_WAIT_NS) return false;
    }
  }
}
// the same without the early exit (draining the CTA's own asynchronous work)
__device__ __forceinline__ bool mbar_drain(uint32_t bar, unsigned parity) {
  unsigned long long t0 = 0;
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 0) {
      const unsigned long long t = gtime();
      if (t0 == 0) t0 = t;
      else if (t - t0 > SK_WAIT_NS) return false;
    }
  }
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
// round to the nearest integer (ties to even), |v| < 2^22
__device__ __forceinline__ float rnd_int(float v) {
  return __fsub_rn(__fadd_rn(v, 12582912.0f), 12582912.0f);
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
__device__ __forceinline__ int exp_above(float mx) {
  if (!(mx > 0.f)) return SK_EXP_MIN;
  const int e = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 126;
  return e < SK_EXP_MIN ? SK_EXP_MIN : (e > SK_EXP_MAX ? SK_EXP_MAX : e);
}

// ------------------------------------------------------ row exponents
// eg[i] = smallest e with |G_ik| < 2^e for all k (rows >= n: the minimum)
__global__ void __launch_bounds__(256)
k_syrk_row_exp(const dd *__restrict__ G, long ldg, int n, int kdim, int *__restrict__ eg, int nrows) {
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  float mx = 0.f;
  if (warp < n) {
    const dd *row = G + (size_t)warp * ldg;
    for (int k = lane; k < kdim; k += 32) mx = fmaxf(mx, fabsf(row[k].hi));
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, m));
  // the low half may lift |G| past the high half's bound by one unit in the
  // last place: bound the sum instead
  if (lane == 0) eg[warp] = warp < n ? exp_above(mx * (1.0f + 1.0f / 1048576.0f)) : SK_EXP_MIN;
}

// ------------------------------------------------------ slices of a k panel
// tiles[T][a][s][128 rows][32 bf16] (64-byte swizzle): rows 128 T .. +127 of
// G, columns k0 + 32 a .. +31 of the panel, slice s.  A 32-row column tile
// J is rows 32 (J mod 4) .. +31 of tile J / 4: 2 KB contiguous per slice.
__global__ void __launch_bounds__(256)
k_syrk_slice(const dd *__restrict__ G, long ldg, int n, int kdim, int k0, const int *__restrict__ eg,
             uint8_t *__restrict__ tiles, int natoms) {
  const int a = blockIdx.x, T = blockIdx.y;
  const int r = threadIdx.x & (SK_TM - 1), h = threadIdx.x >> 7;
  const int i = T * SK_TM + r;
  const int kb = k0 + SK_KA * a + 16 * h;
  const float sc = pow2f(7 - eg[i]);
  float hi[16], lo[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    dd v = dd_zero();
    if (i < n && kb + u < kdim) v = G[(size_t)i * ldg + kb + u];
    hi[u] = v.hi * sc;   // exact: power-of-two scaling
    lo[u] = v.lo * sc;
  }
  uint8_t *base = tiles + ((size_t)T * natoms + a) * SK_NSL * SK_A_SLICE;
#pragma unroll
  for (int s = 0; s < SK_NSL; ++s) {
    uint32_t wd[8];
#pragma unroll
    for (int u2 = 0; u2 < 8; ++u2) {
      float sl[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int u = 2 * u2 + c;
        const float si = rnd_int(hi[u]);
        sl[c] = si * pow2f(-8 * s);
        if (s + 1 < SK_NSL) {
          float rr, ee;
          two_sum(__fsub_rn(hi[u], si), lo[u], rr, ee);   // hi - si is exact
          hi[u] = rr * 256.f;
          lo[u] = ee * 256.f;
        }
      }
      wd[u2] = pack_bf16(sl[0], sl[1]);
    }
    uint8_t *tile = base + (size_t)s * SK_A_SLICE;
    *reinterpret_cast<uint4 *>(tile + swz64(r, 2 * h)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    *reinterpret_cast<uint4 *>(tile + swz64(r, 2 * h + 1)) = make_uint4(wd[4], wd[5], wd[6], wd[7]);
  }
}

// ------------------------------------------ FP64 panels (the Cholesky's updates)
// eg[i] = smallest e with |A_ik| < 2^e over the kdim columns of row i
__global__ void __launch_bounds__(256)
k_syrk_row_exp_d(const double *__restrict__ A, long ld, int n, int kdim, int *__restrict__ eg, int nrows) {
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  double mx = 0.0;
  if (warp < n)
    for (int k = lane; k < kdim; k += 32) mx = fmax(mx, fabs(A[(size_t)warp * ld + k]));
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, m));
  if (lane == 0) {
    int e = SK_EXP_MIN;
    if (warp < n && mx > 0.0) {
      frexp(mx, &e);                    // mx = f 2^e, f in [1/2, 1): mx < 2^e
      e = e < SK_EXP_MIN ? SK_EXP_MIN : (e > SK_EXP_MAX ? SK_EXP_MAX : e);
    }
    eg[warp] = e;
  }
}

// slices of an FP64 panel in the layout of k_syrk_slice: seven 8-bit slices
// hold the 53-bit significand of every entry within 2^2 of its row maximum
// exactly (steps in FP64: scaling by a power of two, rint, and (x - s) 256
// are exact)
__global__ void __launch_bounds__(256)
k_syrk_slice_d(const double *__restrict__ A, long ld, int n, int kdim, const int *__restrict__ eg,
               uint8_t *__restrict__ tiles, int natoms) {
  const int a = blockIdx.x, T = blockIdx.y;
  const int r = threadIdx.x & (SK_TM - 1), h = threadIdx.x >> 7;
  const int i = T * SK_TM + r;
  const int kb = SK_KA * a + 16 * h;
  const int e = eg[i];
  double x[16];
#pragma unroll
  for (int u = 0; u < 16; ++u)
    x[u] = (i < n && kb + u < kdim) ? ldexp(A[(size_t)i * ld + kb + u], 7 - e) : 0.0;
  uint8_t *base = tiles + ((size_t)T * natoms + a) * SK_NSL * SK_A_SLICE;
#pragma unroll
  for (int s = 0; s < SK_NSL; ++s) {
    uint32_t wd[8];
#pragma unroll
    for (int u2 = 0; u2 < 8; ++u2) {
      float sl[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int u = 2 * u2 + c;
        const double si = rint(x[u]);
        sl[c] = (float)si * pow2f(-8 * s);
        x[u] = (x[u] - si) * 256.0;
      }
      wd[u2] = pack_bf16(sl[0], sl[1]);
    }
    uint8_t *tile = base + (size_t)s * SK_A_SLICE;
    *reinterpret_cast<uint4 *>(tile + swz64(r, 2 * h)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    *reinterpret_cast<uint4 *>(tile + swz64(r, 2 * h + 1)) = make_uint4(wd[4], wd[5], wd[6], wd[7]);
  }
}

// pair number p = 0..27 -> (slice of A, slice of B), by level L = 0..6
__device__ __forceinline__ void syrk_pair(int p, int &si, int &sj, int &L) {
  int l = 0, first = 0;
  while (p >= first + l + 1) { first += l + 1; ++l; }
  L = l;
  si = p - first;
  sj = l - si;
}

// ------------------------------------------------------------------ the product
// tile number t: from the list tl, or (tl == nullptr) in row-major order over
// the lower triangle of 128-row tiles, row tile I holding column tiles
// 0 .. 4I+3.  A column tile at or past nc is empty (the last row tile of a
// size that is not a multiple of 128); every role skips it alike.
__device__ __forceinline__ bool tile_at(const int2 *__restrict__ tl, int t, int nc, int2 &out) {
  if (tl) { out = tl[t]; return true; }
  int I = (int)((sqrt(1.0 + 2.0 * (double)t) - 1.0) * 0.5);
  while (2 * (I + 1) * (I + 2) <= t) ++I;
  while (I > 0 && 2 * I * (I + 1) > t) --I;
  out = make_int2(I, t - 2 * I * (I + 1));
  return out.y < nc;
}

// K[i][j] = / += / -= P_ij (mode 0 / 1 / 2) over this panel for the tiles (row
// tile I of 128, column tile J of 32), entries of the lower 64-block triangle
// below n_pad only (n_pad a multiple of 64).
// Warp roles: 0 the bulk-copy issuer, 1 the MMA issuer, 2-5 the epilogue (TMEM
// lane quarter = warp mod 4).  Chunks (SK_CHUNK atoms) alternate between two
// TMEM buffers of SK_NACC x 32 columns.
__global__ void __launch_bounds__(SK_NTHR, 1)
k_syrk_sl(const uint8_t *__restrict__ Sl, const int *__restrict__ eg, const int2 *__restrict__ tl,
          int ntl, int natoms, double *__restrict__ K, long ldk, int n_pad, int mode,
          unsigned tmem_cols, int *err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * SK_S + 5];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int my_tiles = (int)blockIdx.x < ntl ? (ntl - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nchunk = (natoms + SK_CHUNK - 1) / SK_CHUNK;
  const int nc = (n_pad + SK_TN - 1) / SK_TN;
  const uint32_t sbase = (su32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bar0 = su32(&bars[0]);
  auto full = [&](int st) { return bar0 + 8u * st; };
  auto empty = [&](int st) { return bar0 + 8u * (SK_S + st); };
  auto tfull = [&](int bf) { return bar0 + 8u * (2 * SK_S + bf); };
  auto tempty = [&](int bf) { return bar0 + 8u * (2 * SK_S + 2 + bf); };
  const uint32_t drain = bar0 + 8u * (2 * SK_S + 4);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(su32(&tmem_slot)), "r"(tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    fail = 0;
    for (int st = 0; st < SK_S; ++st) {
      mbar_init(full(st), 1);
      mbar_init(empty(st), 1);
    }
    for (int bf = 0; bf < 2; ++bf) {
      mbar_init(tfull(bf), 1);
      mbar_init(tempty(bf), SK_NEPI);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int *vfail = &fail;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- bulk copies: atom a of tile (I, J) into stage st
      int st = 0, use = 0, issued = 0;
      bool ok = true;
      for (int i = 0; i < my_tiles && ok; ++i) {
        int2 t;
        if (!tile_at(tl, (int)blockIdx.x + i * (int)gridDim.x, nc, t)) continue;
        const uint8_t *Abase = Sl + (size_t)t.x * natoms * SK_A_STAGE;
        const uint8_t *Bbase = Sl + (size_t)(t.y >> 2) * natoms * SK_A_STAGE + (size_t)(t.y & 3) * SK_B_SLICE;
        for (int a = 0; a < natoms; ++a) {
          if (use > 0 && !mbar_wait(empty(st), (unsigned)((use - 1) & 1), vfail)) { ok = false; break; }
          const uint32_t dst = sbase + (uint32_t)st * SK_STAGE;
          mbar_arrive_tx(full(st), SK_STAGE);
          bulk_g2s(dst, Abase + (size_t)a * SK_A_STAGE, SK_A_STAGE, full(st));
#pragma unroll
          for (int s = 0; s < SK_NSL; ++s)
            bulk_g2s(dst + SK_A_STAGE + s * SK_B_SLICE, Bbase + (size_t)a * SK_A_STAGE + (size_t)s * SK_A_SLICE,
                     SK_B_SLICE, full(st));
          ++issued;
          if (++st == SK_S) { st = 0; ++use; }
        }
      }
      if (!ok) {
        if (!*vfail && atomicCAS(err, 0, TW_ERR_TIMEOUT) == 0) err[1] = 31;
        fail = 1;
      }
      // copies already issued must land before the CTA's shared memory goes
      if (*vfail)
        for (int a = (issued > SK_S ? issued - SK_S : 0); a < issued; ++a)
          mbar_drain(full(a % SK_S), (unsigned)((a / SK_S) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t idesc = idesc_bf16(SK_TM, SK_TN);
      bool ok = true;
      int st = 0, use = 0, g = 0;                     // stage, its use count, chunk count
      for (int i = 0; i < my_tiles && ok; ++i) {
        int2 t;
        if (!tile_at(tl, (int)blockIdx.x + i * (int)gridDim.x, nc, t)) continue;
        for (int c = 0; c < nchunk && ok; ++c, ++g) {
          const int bf = g & 1;
          // the epilogue has read this buffer's previous chunk
          if (g >= 2 && !mbar_wait(tempty(bf), (unsigned)((g / 2 - 1) & 1), vfail)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dbase = tmem + (uint32_t)(bf * SK_NACC * SK_TN);
          const int a1 = min(natoms, (c + 1) * SK_CHUNK);
          for (int a = c * SK_CHUNK; a < a1; ++a) {
            if (!mbar_wait(full(st), (unsigned)(use & 1), vfail)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aS = sbase + (uint32_t)st * SK_STAGE, bS = aS + SK_A_STAGE;
#pragma unroll
            for (int ks = 0; ks < SK_KA / 16; ++ks) {
#pragma unroll
              for (int p = 0; p < 28; ++p) {
                int si, sj, L;
                syrk_pair(p, si, sj, L);
                const int ac = L < 5 ? L : 5;
                // the first MMA of a chunk into each accumulator overwrites it
                const bool lead = p == 0 || p == 1 || p == 3 || p == 6 || p == 10 || p == 15;
                const uint32_t acc = (a > c * SK_CHUNK || ks > 0 || !lead) ? 1u : 0u;
                mma_bf16(dbase + (uint32_t)(ac * SK_TN), sdesc64(aS + si * SK_A_SLICE + ks * 32),
                         sdesc64(bS + sj * SK_B_SLICE + ks * 32), idesc, acc);
              }
            }
            mma_commit(empty(st));                   // the stage is free once these finish
            if (++st == SK_S) { st = 0; ++use; }
          }
          if (ok) mma_commit(tfull(bf));             // this chunk's sums are final
        }
      }
      if (!ok && !*vfail && atomicCAS(err, 0, TW_ERR_TIMEOUT) == 0) err[1] = 32;
      if (!ok) fail = 1;
      // every issued MMA complete before TMEM is released
      mma_commit(drain);
      mbar_drain(drain, 0);
    }
  } else {
    // ---------------- epilogue: exact level sums into int64, added to K at the end
    const int lg = warp & 3;
    const int r = 32 * lg + lane;
    int g = 0;
    bool ok = true;
    for (int i = 0; i < my_tiles && ok; ++i) {
      int2 t;
      if (!tile_at(tl, (int)blockIdx.x + i * (int)gridDim.x, nc, t)) continue;
      long long T[SK_TN];
      float F[SK_TN];
#pragma unroll
      for (int j = 0; j < SK_TN; ++j) { T[j] = 0; F[j] = 0.f; }
      for (int c = 0; c < nchunk; ++c, ++g) {
        const int bf = g & 1;
        if (!mbar_wait(tfull(bf), (unsigned)((g / 2) & 1), vfail) || *vfail) {
          if (!*vfail && atomicCAS(err, 0, TW_ERR_TIMEOUT) == 0) err[1] = 33;
          fail = 1;
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t trow = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(bf * SK_NACC * SK_TN);
#pragma unroll
        for (int c0 = 0; c0 < SK_TN; c0 += 8) {
          uint32_t d[SK_NACC][8];
#pragma unroll
          for (int ac = 0; ac < SK_NACC; ++ac)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(d[ac][0]), "=r"(d[ac][1]), "=r"(d[ac][2]), "=r"(d[ac][3]), "=r"(d[ac][4]),
                           "=r"(d[ac][5]), "=r"(d[ac][6]), "=r"(d[ac][7])
                         : "r"(trow + (uint32_t)(ac * SK_TN + c0)));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            long long x = __float2int_rn(__uint_as_float(d[0][j]));
#pragma unroll
            for (int L = 1; L < 5; ++L)
              x = x * 256 + __float2int_rn(__uint_as_float(d[L][j]) * pow2f(8 * L));
            T[c0 + j] += x;
            F[c0 + j] += __uint_as_float(d[5][j]);
          }
        }
        // the buffer is read: a later chunk's MMAs may overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(tempty(bf));
      }
      if (!ok) break;
      // a 32-column tile lies inside one 64-block: one mask for the row
      const long row = (long)t.x * SK_TM + r, col0 = (long)t.y * SK_TN;
      if (row < n_pad && col0 < n_pad && (col0 >> 6) <= (row >> 6)) {
        const int ei = eg[row];
        double2 *Kp = reinterpret_cast<double2 *>(K + row * ldk + col0);
        double old[SK_TN];
        if (mode != 0) {
#pragma unroll
          for (int q = 0; q < SK_TN / 2; ++q) {
            const double2 o = Kp[q];
            old[2 * q] = o.x;
            old[2 * q + 1] = o.y;
          }
        }
#pragma unroll
        for (int q = 0; q < SK_TN / 2; ++q) {
          double v[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = 2 * q + h;
            const double p = ldexp((double)T[j] * 0x1p-32 + (double)F[j], ei + eg[col0 + j] - 14);
            v[h] = mode == 0 ? p : (mode == 1 ? old[j] + p : old[j] - p);
          }
          Kp[q] = make_double2(v[0], v[1]);
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
// the lower 64-block triangle as (128-row tile, 32-column tile): groups of 8
// row tiles, column tile outer, row tile inner
void syrk_tile_list(int n_pad, std::vector<int2> &tl) {
  const int nt = (n_pad + SK_TM - 1) / SK_TM, nc = (n_pad + SK_TN - 1) / SK_TN;
  tl.clear();
  for (int g0 = 0; g0 < nt; g0 += 8) {
    const int g1 = std::min(nt, g0 + 8);
    const int jmax = std::min(nc - 1, 4 * (g1 - 1) + 3);
    for (int J = 0; J <= jmax; ++J)
      for (int I = g0; I < g1; ++I)
        if (J <= 4 * I + 3) tl.push_back(make_int2(I, J));
  }
}

size_t syrk_ws_bytes_per_atom(int n_pad) {
  return (size_t)((n_pad + SK_TM - 1) / SK_TM) * SK_A_STAGE;
}
int syrk_exp_rows(int n_pad) { return (n_pad + SK_TM - 1) / SK_TM * SK_TM; }

// K[i][j] = (G G^T)_ij for the lower 64-block triangle of the n_pad x n_pad
// array K (rows of G >= n are zero); ws holds one panel of slices (a multiple
// of syrk_ws_bytes_per_atom), eg syrk_exp_rows(n_pad) ints, tl the tile list
cudaError_t launch_form_P_tc(const dd *G, long ldg, int n, int kdim, double *K, long ldk, int n_pad,
                             uint8_t *ws, size_t ws_bytes, int *eg, const int2 *tl, int ntl, int *err,
                             cudaStream_t s) {
  if (n <= 0 || n_pad <= 0 || ntl <= 0) return cudaSuccess;
  const int nt = (n_pad + SK_TM - 1) / SK_TM, nrows = nt * SK_TM;
  k_syrk_row_exp<<<(unsigned)(((long)nrows * 32 + 255) / 256), 256, 0, s>>>(G, ldg, n, kdim, eg, nrows);
  count_launches(1);
  const int atoms_total = (kdim + SK_KA - 1) / SK_KA;
  int per_panel = (int)std::min<size_t>(ws_bytes / syrk_ws_bytes_per_atom(n_pad), (size_t)atoms_total);
  if (per_panel > SK_CHUNK) per_panel -= per_panel % SK_CHUNK;
  if (per_panel < 1) return cudaErrorInvalidValue;
  const size_t sm = (size_t)SK_S * SK_STAGE + 1024;
  cudaFuncSetAttribute(k_syrk_sl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::max(1, std::min(ntl, nsm));
  for (int a0 = 0; a0 < atoms_total; a0 += per_panel) {
    const int na = std::min(per_panel, atoms_total - a0);
    k_syrk_slice<<<dim3((unsigned)na, (unsigned)nt), 256, 0, s>>>(G, ldg, n, kdim, a0 * SK_KA, eg, ws, na);
    count_launches(1);
    k_syrk_sl<<<grid, SK_NTHR, sm, s>>>(ws, eg, tl, ntl, na, K, ldk, n_pad, a0 == 0 ? 0 : 1, 512u, err);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// C -= A A^T for the lower 64-block triangle of the m x m array C (row
// stride ldc; m a multiple of 64), A the m x kdim FP64 panel (row stride lda,
// kdim a multiple of 32): the blocked Cholesky's trailing update, exact
// products on the tensor cores.  ws >= syrk_ws_bytes_per_atom(m) * kdim / 32
// bytes, eg >= syrk_exp_rows(m) ints.
cudaError_t launch_syrk_update_d(const double *A, long lda, int kdim, double *C, long ldc, int m,
                                 uint8_t *ws, size_t ws_bytes, int *eg, int *err, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int natoms = kdim / SK_KA;
  if (m % 64 != 0 || kdim % SK_KA != 0 || natoms < 1 || ws_bytes < syrk_ws_bytes_per_atom(m) * natoms)
    return cudaErrorInvalidValue;
  const int nt = (m + SK_TM - 1) / SK_TM, nrows = nt * SK_TM;
  k_syrk_row_exp_d<<<(unsigned)(((long)nrows * 32 + 255) / 256), 256, 0, s>>>(A, lda, m, kdim, eg, nrows);
  count_launches(1);
  k_syrk_slice_d<<<dim3((unsigned)natoms, (unsigned)nt), 256, 0, s>>>(A, lda, m, kdim, eg, ws, natoms);
  count_launches(1);
  const size_t sm = (size_t)SK_S * SK_STAGE + 1024;
  cudaFuncSetAttribute(k_syrk_sl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int ntl = 2 * nt * (nt + 1);                 // closed-form row-major order
  const unsigned grid = (unsigned)std::max(1, std::min(ntl, nsm));
  k_syrk_sl<<<grid, SK_NTHR, sm, s>>>(ws, eg, nullptr, ntl, natoms, C, ldc, m, 2, 512u, err);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tw
