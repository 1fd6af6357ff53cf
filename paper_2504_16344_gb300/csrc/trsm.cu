// trsm.cu -- triangular solves with K's factor for a batch of right-hand
// sides, each with its own observation window.
//
// The online solve K' y = d (Sec. "Real-time inference", the data-space
// form of the posterior mean) for a window of Nt' steps uses the leading
// n' = Nd Nt' rows and columns of the factor L, because the leading block of
// K is the windowed K and Cholesky factors nest.  For B right-hand sides
// the sweeps
//   forward  L Z = D,   backward  L^T Y = Z
// become block products L_IJ (64x64) x Z_J (64 x CS): the factor block is
// read once per column slice of CS right-hand sides instead of once per
// right-hand side.
//
// Scheduling (one persistent kernel per sweep): a ticket counter hands out
// (block row, column slice) pairs in block-row order; each slice keeps its
// own progress counter (rows finished, in dependency order), so slices
// advance independently.  A slice's active block rows are those below the
// largest window among its columns; rows past it are written as zero and
// take no part in the dependency chain.  In a row, every dependency but
// the last is summed as soon as it is ready (factor blocks streamed into
// shared memory with asynchronous copies, double-buffered); the diagonal
// inverse is applied before waiting for the last one, which costs a single
// 64x64 product with the precomputed chain block.  Every wait is bounded
// (2 s), after which the kernel records TW_ERR_TIMEOUT, raises the abort
// flag that all CTAs poll, and returns.
//
// Element types: double (native FP64, with L itself: the QoI set-up) and dd
// (float pairs, with the single-vector solve's blocks pre-multiplied by the
// diagonal-block inverses: the online batched solves of every precision path,
// in double-float arithmetic on the FP32 pipes, like the single-vector solve).
#include <algorithm>

#include "../../include/tw.h"
#include "dense_api.h"
#include "kernels.h"

namespace tw {

namespace {

constexpr int CS = 8;      // right-hand sides per column slice
constexpr int LDA = 66;    // padded row stride (elements) of shared 64x64 tiles
constexpr int LDZ = 66;    // padded column stride of shared 64 x CS tiles
constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acq(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void note_error(int *err, int code, int info) {
  if (atomicCAS(err, 0, code) == 0) err[1] = info;
}

// 16-byte asynchronous copy global -> shared, cached in L2 only
__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// one 64x64 block (8-byte elements, rows contiguous) into a padded shared tile
template <class T>
__device__ __forceinline__ void stage_block(T *dst, const T *__restrict__ src) {
  // 64 rows x 32 sixteen-byte pieces = 2048 pieces, 8 per thread
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int p = threadIdx.x + 256 * i;
    const int row = p >> 5, piece = p & 31;
    cp16(dst + row * LDA + piece * 2, src + row * NB_ + piece * 2);
  }
}

// the slice's CS columns of dependency block J (written by other CTAs) into a
// shared 64 x CS tile: one 16-byte piece per thread, L2 only, zeros for
// columns past the batch
template <class T>
__device__ __forceinline__ void stage_z(T *Zd, const T *__restrict__ out, long out_bstride, int b0,
                                        int B, int J) {
  static_assert(sizeof(T) == 8, "8-byte elements");
  static_assert(CS * NB_ / 2 == 256, "one piece per thread");
  const int c = threadIdx.x >> 5, piece = threadIdx.x & 31;
  const bool ok = b0 + c < B;
  const T *src = ok ? out + (long)(b0 + c) * out_bstride + (long)J * NB_ + 2 * piece : out;
  const unsigned sa = (unsigned)__cvta_generic_to_shared(Zd + c * LDZ + 2 * piece);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(src), "r"(ok ? 16 : 0) : "memory");
}

template <class T> struct TS;
template <> struct TS<double> {
  typedef double acc;
  static __device__ __forceinline__ acc zero() { return 0.0; }
  static __device__ __forceinline__ void mac(acc &a, double x, double y) { a = fma(x, y, a); }
  static __device__ __forceinline__ double get(acc a) { return a; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double zv() { return 0.0; }
  static __device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
  static __device__ __forceinline__ double ld_rhs(const void *p, int kind, long i) {
    if (kind == 0) return __ldcg(reinterpret_cast<const double *>(p) + i);
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p) + i);
    return (double)v.x + (double)v.y;
  }
};
template <> struct TS<dd> {
  typedef dacc acc;
  static __device__ __forceinline__ acc zero() { return dacc_zero(); }
  static __device__ __forceinline__ void mac(acc &a, dd x, dd y) { dacc_mac(a, x, y); }
  static __device__ __forceinline__ dd get(acc a) { return dacc_get(a); }
  static __device__ __forceinline__ dd sub(dd a, dd b) { return dd_sub(a, b); }
  static __device__ __forceinline__ dd zv() { return dd_zero(); }
  static __device__ __forceinline__ dd ld_cg(const dd *p) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    dd r; r.hi = v.x; r.lo = v.y; return r;
  }
  static __device__ __forceinline__ dd ld_rhs(const void *p, int kind, long i) {
    if (kind == 0) return dd_from_double(__ldcg(reinterpret_cast<const double *>(p) + i));
    return ld_cg(reinterpret_cast<const dd *>(p) + i);
  }
};

// acc[j] += sum_k A(r, k) V[c_j][k] with A(r, k) = A[r][k] (FWD) or A[k][r] (BWD)
template <class T, bool FWD>
__device__ __forceinline__ void tile_mac(typename TS<T>::acc *acc, const T *A, const T *V, int r,
                                         int c0) {
  typedef TS<T> S;
  const T *v0 = V + c0 * LDZ, *v1 = V + (c0 + 1) * LDZ;
#pragma unroll 16
  for (int k = 0; k < NB_; ++k) {
    const T a = FWD ? A[r * LDA + k] : A[k * LDA + r];
    S::mac(acc[0], a, v0[k]);
    S::mac(acc[1], a, v1[k]);
  }
}

// SCALED: Lp holds the factor's blocks pre-multiplied by the diagonal-block
// inverses, Lf_IJ = Linv_I L_IJ (FWD) or Lb_IJ = L_IJ Linv_J (BWD), so that
//   z_I = Linv_I d_I - sum_J<I Lf_IJ z_J,   y_J = Linv_J^T z_J - sum_I>J Lb_IJ^T y_I;
// the diagonal inverse then multiplies the right-hand side alone and the last
// dependency's block is its own chain block (Lchain is not used).
template <class T, bool FWD, bool SCALED>
__global__ void __launch_bounds__(256, 2)
k_trsm(const T *__restrict__ Lp, const T *__restrict__ Linv, const T *__restrict__ Lchain,
       const void *__restrict__ rhs, int rhs_kind, long rhs_bstride, T *__restrict__ out,
       long out_bstride, const int *__restrict__ win, int Nd, int Nt, int B, int NB, int nslices,
       int *prog, int *err, int *abort_flag) {
  typedef TS<T> S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *As = reinterpret_cast<T *>(smem_raw);   // [2][64][LDA]
  T *Zs = As + 2 * NB_ * LDA;                 // [2][CS][LDZ]
  T *Vs = Zs + 2 * CS * LDZ;                  // [CS][LDZ]
  __shared__ int sT, sP, sbail;
  const int tid = threadIdx.x;
  const int r = tid >> 2, c0 = 2 * (tid & 3);
  const long ntickets = (long)NB * nslices;
  for (;;) {
    __syncthreads();   // everyone has read the previous ticket
    if (tid == 0) { sT = atomicAdd(prog, 1); sbail = 0; }
    __syncthreads();
    const int t = sT;
    if (t >= ntickets) return;
    const int It = t / nslices, sl = t % nslices;
    const int I = FWD ? It : NB - 1 - It;
    const int b0 = sl * CS;
    // rows of every column of the slice; the slice's active block rows
    int nrows[2] = {0, 0};
    int nmax = 0;
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      const int b = b0 + c;
      const int nr = b < B ? Nd * min(max(__ldg(win + b), 0), Nt) : 0;
      nmax = max(nmax, nr);
      if (c == c0) nrows[0] = nr;
      if (c == c0 + 1) nrows[1] = nr;
    }
    const int NBs = (nmax + NB_ - 1) / NB_;
    const long gi = (long)I * NB_ + r;
    T *o0 = out + (long)(b0 + c0) * out_bstride;
    T *o1 = o0 + out_bstride;
    const bool has0 = b0 + c0 < B, has1 = b0 + c0 + 1 < B;
    if (I >= NBs) {                      // past every window of the slice
      if (has0) o0[gi] = S::zv();
      if (has1) o1[gi] = S::zv();
      continue;
    }
    const int u = FWD ? I : NBs - 1 - I;   // position in the slice's dependency order
    int *progress = prog + 1 + sl;
    T bv[2];
    bv[0] = (has0 && gi < nrows[0]) ? S::ld_rhs(rhs, rhs_kind, (long)(b0 + c0) * rhs_bstride + gi) : S::zv();
    bv[1] = (has1 && gi < nrows[1]) ? S::ld_rhs(rhs, rhs_kind, (long)(b0 + c0 + 1) * rhs_bstride + gi) : S::zv();
    // ---- bulk: dependencies 0 .. u-2 (block J = d for FWD, NBs-1-d for BWD)
    typename S::acc acc[2] = {S::zero(), S::zero()};
    const int nbulk = u > 0 ? u - 1 : 0;
    auto dep_block = [&](int d) -> const T * {
      const int J = FWD ? d : NBs - 1 - d;
      return Lp + (FWD ? packed_index(I, J) : packed_index(J, I)) * NB_ * NB_;
    };
    if (nbulk > 0) { stage_block(As, dep_block(0)); cp_commit(); }
    int d = 0;
    bool zpre = false;   // Z of dependency d already requested
    while (d < nbulk) {
      if (tid == 0) {
        int p = ld_acq(progress);
        if (p <= d) {
          const unsigned long long t0 = now_ns();
          while ((p = ld_acq(progress)) <= d) {
            if (*(volatile int *)abort_flag) { sbail = 1; break; }
            if (now_ns() - t0 > WAIT_NS) {
              note_error(err, TW_ERR_TIMEOUT, FWD ? 5 : 6);
              atomicExch(abort_flag, 1);
              sbail = 1;
              break;
            }
            const int behind = u - p;
            __nanosleep(behind > 2 ? min(4096, 256 * (behind - 2)) : 64);
          }
        }
        sP = p;
      }
      __syncthreads();
      if (sbail) { cp_wait<0>(); return; }
      const int dend = min(sP, nbulk);
      // dependency values Z_J (written by other CTAs) are copied like the
      // factor blocks: a dependency known to be ready has its Z requested in
      // the same group as its block, one step ahead of its product
      if (!zpre && d < dend) {
        stage_z(Zs + (d & 1) * CS * LDZ, out, out_bstride, b0, B, FWD ? d : NBs - 1 - d);
        cp_commit();
        zpre = true;
      }
      for (; d < dend; ++d) {
        bool znext = false;
        if (d + 1 < nbulk) {
          stage_block(As + ((d + 1) & 1) * NB_ * LDA, dep_block(d + 1));
          if (d + 1 < dend) {
            stage_z(Zs + ((d + 1) & 1) * CS * LDZ, out, out_bstride, b0, B, FWD ? d + 1 : NBs - 2 - d);
            znext = true;
          }
          cp_commit();
          cp_wait<1>();   // all but the newest group: block d and Z_d are in
        } else {
          cp_wait<0>();
        }
        __syncthreads();
        tile_mac<T, FWD>(acc, As + (d & 1) * NB_ * LDA, Zs + (d & 1) * CS * LDZ, r, c0);
        __syncthreads();
        zpre = znext;
      }
    }
    // ---- v = b - bulk;  w = Linv v (FWD) or Linv^T v (BWD)
    //      (SCALED: v = b, and the bulk is subtracted from w)
    stage_block(As, Linv + (size_t)I * NB_ * NB_);
    cp_commit();
    const bool chain = u > 0;
    if (chain) {
      stage_block(As + NB_ * LDA, SCALED ? dep_block(u - 1) : Lchain + (size_t)I * NB_ * NB_);
      cp_commit();
    }
    if constexpr (SCALED) {
      Vs[c0 * LDZ + r] = (gi < nrows[0]) ? bv[0] : S::zv();
      Vs[(c0 + 1) * LDZ + r] = (gi < nrows[1]) ? bv[1] : S::zv();
    } else {
      Vs[c0 * LDZ + r] = (gi < nrows[0]) ? S::sub(bv[0], S::get(acc[0])) : S::zv();
      Vs[(c0 + 1) * LDZ + r] = (gi < nrows[1]) ? S::sub(bv[1], S::get(acc[1])) : S::zv();
    }
    if (chain) cp_wait<1>(); else cp_wait<0>();
    __syncthreads();
    typename S::acc wacc[2] = {S::zero(), S::zero()};
    tile_mac<T, FWD>(wacc, As, Vs, r, c0);
    T res[2] = {S::get(wacc[0]), S::get(wacc[1])};
    if constexpr (SCALED) {
      res[0] = S::sub(res[0], S::get(acc[0]));
      res[1] = S::sub(res[1], S::get(acc[1]));
    }
    // ---- the last dependency: one product with the chain block
    if (chain) {
      if (tid == 0) {
        const unsigned long long t0 = now_ns();
        while (ld_acq(progress) < u) {
          if (*(volatile int *)abort_flag) { sbail = 1; break; }
          if (now_ns() - t0 > WAIT_NS) {
            note_error(err, TW_ERR_TIMEOUT, FWD ? 7 : 8);
            atomicExch(abort_flag, 1);
            sbail = 1;
            break;
          }
          __nanosleep(32);
        }
      }
      __syncthreads();
      if (sbail) { cp_wait<0>(); return; }
      const int J = FWD ? I - 1 : I + 1;
      for (int i = tid; i < CS * NB_; i += 256) {
        const int c = i >> 6, k = i & 63;
        Zs[c * LDZ + k] = (b0 + c < B) ? S::ld_cg(out + (long)(b0 + c) * out_bstride + (long)J * NB_ + k)
                                       : S::zv();
      }
      cp_wait<0>();
      __syncthreads();
      typename S::acc cacc[2] = {S::zero(), S::zero()};
      tile_mac<T, FWD>(cacc, As + NB_ * LDA, Zs, r, c0);
      res[0] = S::sub(res[0], S::get(cacc[0]));
      res[1] = S::sub(res[1], S::get(cacc[1]));
    }
    if (has0) o0[gi] = gi < nrows[0] ? res[0] : S::zv();
    if (has1) o1[gi] = gi < nrows[1] ? res[1] : S::zv();
    __syncthreads();   // every store before thread 0's (cumulative) release
    if (tid == 0) st_rel(progress, u + 1);
  }
}

template <class T, bool SCALED>
cudaError_t trsm(const T *Lp, const T *Linv, const T *Lchain, const void *rhs, int rhs_kind,
                 long rhs_bstride, T *out, long out_bstride, const int *win, int Nd, int Nt, int B,
                 int NB, int *prog, bool fwd, int *err, int *abort_flag, cudaStream_t s) {
  if (B <= 0 || NB <= 0) return cudaSuccess;
  const int nslices = (B + CS - 1) / CS;
  cudaError_t e = cudaMemsetAsync(prog, 0, sizeof(int) * (1 + nslices), s);
  if (e != cudaSuccess) return e;
  const size_t sm = sizeof(T) * (2 * NB_ * LDA + 3 * CS * LDZ);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long tickets = (long)NB * nslices;
  const int grid = (int)std::min<long>(tickets, 2L * nsm);
  if (fwd) {
    cudaFuncSetAttribute(k_trsm<T, true, SCALED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_trsm<T, true, SCALED><<<grid, 256, sm, s>>>(Lp, Linv, Lchain, rhs, rhs_kind, rhs_bstride, out,
                                          out_bstride, win, Nd, Nt, B, NB, nslices, prog, err,
                                          abort_flag);
  } else {
    cudaFuncSetAttribute(k_trsm<T, false, SCALED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_trsm<T, false, SCALED><<<grid, 256, sm, s>>>(Lp, Linv, Lchain, rhs, rhs_kind, rhs_bstride, out,
                                           out_bstride, win, Nd, Nt, B, NB, nslices, prog, err,
                                           abort_flag);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

int trsm_prog_ints(int B) { return 1 + (B + CS - 1) / CS; }

cudaError_t launch_trsm_d(const double *Lp, const double *Linv, const double *Lchain,
                          const void *rhs, int rhs_kind, long rhs_bstride, double *out,
                          long out_bstride, const int *win, int Nd, int Nt, int B, int NB,
                          int *prog, bool fwd, int *err, int *abort_flag, cudaStream_t s) {
  return trsm<double, false>(Lp, Linv, Lchain, rhs, rhs_kind, rhs_bstride, out, out_bstride, win, Nd, Nt,
                             B, NB, prog, fwd, err, abort_flag, s);
}
cudaError_t launch_trsm_dd_scaled(const dd *Lx, const dd *Linv, const void *rhs, int rhs_kind,
                                  long rhs_bstride, dd *out, long out_bstride, const int *win, int Nd,
                                  int Nt, int B, int NB, int *prog, bool fwd, int *err, int *abort_flag,
                                  cudaStream_t s) {
  return trsm<dd, true>(Lx, Linv, nullptr, rhs, rhs_kind, rhs_bstride, out, out_bstride, win, Nd, Nt, B,
                        NB, prog, fwd, err, abort_flag, s);
}

}  // namespace tw
