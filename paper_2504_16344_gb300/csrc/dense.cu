#include <algorithm>
// dense.cu -- the data-space Hessian K: formation, Cholesky, triangular solves.
//
// Phase 2 of the paper forms K = Gamma_n + F Gamma_pr F* and Cholesky-factors
// it; Phase 4 solves K y = d online (Sec. "Real-time Bayesian inference and
// prediction framework").  Here K is formed from the time-domain block
// column without unit-vector applies: with Phi the (Nd Nt) x Nm matrix whose
// row block u is F_u and G = Phi C^{1/2},
//   P = G G^T,  K_(i,j) = sigma^2 delta_ij I + sum_{s<=min(i,j)} P_(i-s, j-s),
// i.e. a symmetric rank-Nm product (on the tensor cores, gemm_syrk.cu)
// followed by prefix sums along the Nd x Nd block diagonals (time-major
// ordering, as in the paper's data vectors).
//
// All matrices use 64 x 64 tiles.  K is held in full (lower triangle used)
// with leading dimension n_pad = 64 * ceil(n/64); the padding has an
// identity diagonal so every tile is full.  The factor is then packed as
// lower-triangular 64 x 64 blocks (block (I,J) at I(I+1)/2 + J), contiguous
// for streaming, plus explicit inverses of the diagonal blocks.
//
// Triangular solves run as one persistent launch: CTAs take block rows in
// order from an atomic ticket, stream their off-diagonal blocks while
// waiting for the blocks they depend on (a flag per block row, released
// after the block's result is stored), and finish with the inverted
// diagonal block.  A CTA only waits on rows with earlier tickets, which are
// held by CTAs already running, so the launch cannot deadlock; every wait is
// bounded in time and reports TW_ERR_TIMEOUT instead of hanging.
#include "../../include/tw.h"
#include "dense.cuh"
#include "dense_api.h"
#include "kernels.h"

namespace tw {

namespace {

template <class T> __device__ __forceinline__ T ldT(const T *p) { return *p; }

__device__ __forceinline__ void record_error(int *err, int code, int info) {
  if (atomicCAS(err, 0, code) == 0) atomicExch(err + 1, info);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class T> __device__ __forceinline__ T ld_cg(const T *p);
template <> __device__ __forceinline__ dd ld_cg<dd>(const dd *p) {
  float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  dd r; r.hi = v.x; r.lo = v.y; return r;
}
template <> __device__ __forceinline__ float ld_cg<float>(const float *p) { return __ldcg(p); }

// -------------------------------------------------------------- GEMM NT
// C[tile (I,J)] = (subtract ? C - S : S),  S = sum_k A[i][k] B[j][k]
// A rows >= arows and B rows >= brows are zero.  lower: skip J > I.
// Products accumulate in T over runs of 32 and the run sums are added into
// totals of type TC (the Cholesky's trailing updates: TC = T).
template <class T, class TC> struct Fold;
template <class T> struct Fold<T, T> {
  static __device__ __forceinline__ void run(T &tot, typename DS<T>::acc &a) { DS<T>::fold(tot, a); }
};

template <class T, class TC = T>
__global__ void __launch_bounds__(256)
k_gemm_nt(const T *__restrict__ A, long lda, int arows, const T *__restrict__ B, long ldb,
          int brows, int kdim, TC *__restrict__ C, long ldc, int lower, int subtract) {
  typedef DS<T> S;
  constexpr int KC = 16;
  __shared__ T As[KC][NB_ + 4];
  __shared__ T Bs[KC][NB_ + 4];
  const int I = blockIdx.y, J = blockIdx.x;
  if (lower && J > I) return;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  typename S::acc acc[4][4];
  TC tot[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) { acc[u][v] = S::zero(); tot[u][v] = DS<TC>::zerov(); }
  const int lr = tid >> 2, lk = (tid & 3) * 4;   // loader: row, first k
  const long arow = (long)I * NB_ + lr, brow = (long)J * NB_ + lr;
  for (int k0 = 0; k0 < kdim; k0 += KC) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + lk + q;
      As[lk + q][lr] = (arow < arows && k < kdim) ? A[arow * lda + k] : S::zerov();
      Bs[lk + q][lr] = (brow < brows && k < kdim) ? B[brow * ldb + k] : S::zerov();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty * 4 + u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx * 4 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) S::mac(acc[u][v], a[u], b[v]);
    }
    // fold the compensated chunk sums into the running totals every 32
    // products (and after the last chunk)
    if (((k0 / KC) & 1) || k0 + KC >= kdim) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) Fold<T, TC>::run(tot[u][v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long i = (long)I * NB_ + ty * 4 + u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long j = (long)J * NB_ + tx * 4 + v;
      TC s = tot[u][v];
      C[i * ldc + j] = subtract ? DS<TC>::sub(C[i * ldc + j], s) : s;
    }
  }
}

// ------------------------------------------- K from P: block-diagonal prefix
// K[(t+delta)Nd + a][t Nd + b] += K[(t+delta-1)Nd + a][(t-1)Nd + b], t = 1..Nt-1-delta
__global__ void k_prefix_diag(double *__restrict__ K, long ldk, int Nd, int Nt) {
  const long per = (long)Nd * Nd;
  const long total = (long)Nt * per;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const int delta = (int)(idx / per);
    const int a = (int)((idx % per) / Nd), b = (int)(idx % Nd);
    if (delta == 0 && b > a) continue;
    double run = ldT(K + ((long)delta * Nd + a) * ldk + b);   // t = 0 term
    for (int t = 1; t + delta < Nt; ++t) {
      double *p = K + ((long)(t + delta) * Nd + a) * ldk + (long)t * Nd + b;
      run += *p;
      *p = run;
    }
  }
}

// diagonal: += sigma^2 inside, 1 on the padding
__global__ void k_diag_set(double *__restrict__ K, long ldk, int n, int n_pad, double s2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  double *p = K + (long)i * ldk + i;
  *p = (i < n) ? *p + s2 : 1.0;
}

// ----------------------------------------------- Cholesky: diagonal block
// Factors the 64x64 diagonal block J in place (lower) and writes the inverse
// of the factor block to inv ([64][64], upper part zero).
template <class T>
__global__ void __launch_bounds__(256)
k_potrf_diag(T *__restrict__ K, long ldk, int J, T *__restrict__ inv, int *err) {
  typedef DS<T> S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*sA)[NB_ + 1] = reinterpret_cast<T(*)[NB_ + 1]>(smem_raw);
  T(*sX)[NB_ + 1] = sA + NB_;
  __shared__ T sInv[NB_];
  const int tid = threadIdx.x;
  T *Ablk = K + (long)J * NB_ * ldk + (long)J * NB_;
  for (int idx = tid; idx < NB_ * NB_; idx += blockDim.x) {
    const int r = idx / NB_, c = idx % NB_;
    sA[r][c] = (c <= r) ? Ablk[(long)r * ldk + c] : S::zerov();
  }
  __syncthreads();
  for (int c = 0; c < NB_; ++c) {
    if (tid == 0) {
      T piv = sA[c][c];
      if (!(S::lead(piv) > 0)) {   // not positive definite (or NaN)
        record_error(err, TW_ERR_NOT_SPD, J * NB_ + c);
        piv = S::one();
      }
      const T d = S::sqrtv(piv);
      sA[c][c] = d;
      sInv[c] = S::div(S::one(), d);
    }
    __syncthreads();
    for (int r = c + 1 + tid; r < NB_; r += blockDim.x) sA[r][c] = S::mul(sA[r][c], sInv[c]);
    __syncthreads();
    const int m = NB_ - 1 - c;
    const int ntri = m * (m + 1) / 2;
    for (int idx = tid; idx < ntri; idx += blockDim.x) {
      int rr = (int)((sqrtf(8.f * idx + 1.f) - 1.f) * 0.5f);
      while (rr * (rr + 1) / 2 > idx) --rr;
      while ((rr + 1) * (rr + 2) / 2 <= idx) ++rr;
      const int kk = idx - rr * (rr + 1) / 2;
      const int r = c + 1 + rr, k = c + 1 + kk;
      typename S::acc a = S::zero();
      S::mac(a, S::neg(sA[r][c]), sA[k][c]);
      sA[r][k] = S::add(sA[r][k], S::get(a));
    }
    __syncthreads();
  }
  // write the factor block back (lower part)
  for (int idx = tid; idx < NB_ * NB_; idx += blockDim.x) {
    const int r = idx / NB_, c = idx % NB_;
    if (c <= r) Ablk[(long)r * ldk + c] = sA[r][c];
  }
  // inverse by forward substitution, one column per thread: L X = I
  if (tid < NB_) {
    const int j = tid;
    for (int r = 0; r < j; ++r) sX[r][j] = S::zerov();
    sX[j][j] = sInv[j];
    for (int r = j + 1; r < NB_; ++r) {
      typename S::acc a = S::zero();
      T t = S::zerov();
      for (int k = j; k < r; ++k) {
        S::mac(a, sA[r][k], sX[k][j]);
        if (((k - j) & 15) == 15) S::fold(t, a);
      }
      S::fold(t, a);
      sX[r][j] = S::neg(S::mul(t, sInv[r]));
    }
  }
  __syncthreads();
  for (int idx = tid; idx < NB_ * NB_; idx += blockDim.x) {
    const int r = idx / NB_, c = idx % NB_;
    inv[idx] = sX[r][c];
  }
}

// ---------------------------------------- Cholesky: panel (substitution)
// rows of block I = J+1+blockIdx.x: X L_JJ^T = A_IJ  (one row per thread)
template <class T>
__global__ void __launch_bounds__(64)
k_trsm_panel(T *__restrict__ K, long ldk, int J) {
  typedef DS<T> S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*sL)[NB_ + 1] = reinterpret_cast<T(*)[NB_ + 1]>(smem_raw);
  T(*sX)[NB_ + 1] = sL + NB_;
  __shared__ T sInv[NB_];
  const int tid = threadIdx.x;
  const int I = J + 1 + blockIdx.x;
  const T *Lblk = K + (long)J * NB_ * ldk + (long)J * NB_;
  T *Ablk = K + (long)I * NB_ * ldk + (long)J * NB_;
  for (int idx = tid; idx < NB_ * NB_; idx += blockDim.x) {
    const int r = idx / NB_, c = idx % NB_;
    sL[r][c] = (c <= r) ? Lblk[(long)r * ldk + c] : S::zerov();
    sX[r][c] = Ablk[(long)r * ldk + c];
  }
  __syncthreads();
  sInv[tid] = S::div(S::one(), sL[tid][tid]);
  __syncthreads();
  const int r = tid;
  for (int c = 0; c < NB_; ++c) {
    typename S::acc a = S::zero();
    T t = S::zerov();
    for (int k = 0; k < c; ++k) {
      S::mac(a, sX[r][k], sL[c][k]);
      if ((k & 15) == 15) S::fold(t, a);
    }
    S::fold(t, a);
    sX[r][c] = S::mul(S::sub(sX[r][c], t), sInv[c]);
  }
  __syncthreads();
  for (int idx = tid; idx < NB_ * NB_; idx += blockDim.x) {
    const int rr = idx / NB_, c = idx % NB_;
    Ablk[(long)rr * ldk + c] = sX[rr][c];
  }
}

// ---------------------------------------------------------- packing
template <class T>
__global__ void k_pack(const T *__restrict__ K, long ldk, T *__restrict__ P, int NB) {
  const size_t nblk = (size_t)NB * (NB + 1) / 2;
  for (size_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    int I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((size_t)I * (I + 1) / 2 > b) --I;
    while ((size_t)(I + 1) * (I + 2) / 2 <= b) ++I;
    const int J = (int)(b - (size_t)I * (I + 1) / 2);
    const T *src = K + (long)I * NB_ * ldk + (long)J * NB_;
    T *dst = P + b * NB_ * NB_;
    for (int idx = threadIdx.x; idx < NB_ * NB_; idx += blockDim.x) {
      const int r = idx / NB_, c = idx % NB_;
      dst[idx] = (I == J && c > r) ? DS<T>::zerov() : src[(long)r * ldk + c];
    }
  }
}

// packed blocks of a double factor -> dd packed blocks (hi = rn(x), lo = rn(x - hi))
__global__ void k_double_to_dd(const double *__restrict__ a, dd *__restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = dd_from_double(a[i]);
}

// pack lower blocks of a double matrix into dd packed blocks
__global__ void k_pack_d2dd(const double *__restrict__ K, long ldk, dd *__restrict__ P, int NB) {
  const size_t nblk = (size_t)NB * (NB + 1) / 2;
  for (size_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    int I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((size_t)I * (I + 1) / 2 > b) --I;
    while ((size_t)(I + 1) * (I + 2) / 2 <= b) ++I;
    const int J = (int)(b - (size_t)I * (I + 1) / 2);
    const double *src = K + (long)I * NB_ * ldk + (long)J * NB_;
    dd *dst = P + b * NB_ * NB_;
    for (int idx = threadIdx.x; idx < NB_ * NB_; idx += blockDim.x) {
      const int r = idx / NB_, c = idx % NB_;
      dst[idx] = (I == J && c > r) ? dd_zero() : dd_from_double(src[(long)r * ldk + c]);
    }
  }
}

// full dd matrix (lower tiles) -> float
__global__ void k_lower_to_float(const double *__restrict__ K, float *__restrict__ K32, long ld, int NB) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (J > I) return;
  for (int idx = threadIdx.x; idx < NB_ * NB_; idx += blockDim.x) {
    const int r = idx / NB_, c = idx % NB_;
    const long o = ((long)I * NB_ + r) * ld + (long)J * NB_ + c;
    K32[o] = __double2float_rn(K[o]);
  }
}

// ------------------------------------------------------ triangular solves
// FWD: L z = b (b from `rhs`, rows >= nrows zero);  BWD: L^T x = z.
// Lp: packed blocks; Linv: [NB][64][64] inverses of the diagonal blocks.
template <class T> __device__ __forceinline__ T ld_rhs(const void *rhs, int kind, long i);
template <> __device__ __forceinline__ float ld_rhs<float>(const void *rhs, int kind, long i) {
  if (kind == 0) return __double2float_rn(reinterpret_cast<const double *>(rhs)[i]);
  if (kind == 1) { dd v = ld_cg(reinterpret_cast<const dd *>(rhs) + i); return __fadd_rn(v.hi, v.lo); }
  return __ldcg(reinterpret_cast<const float *>(rhs) + i);
}

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s

template <class T> __device__ __forceinline__ T ldg_t(const T *p);
template <> __device__ __forceinline__ float ldg_t<float>(const float *p) { return __ldg(p); }

// 16 consecutive elements of T from 16-byte-aligned storage, as vector loads
// (elements assigned one by one so the array stays in registers)
template <class T> __device__ __forceinline__ void ld16(const T *__restrict__ p, T *v);
template <> __device__ __forceinline__ void ld16<float>(const float *__restrict__ p, float *v) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 t = __ldg(q + i);
    v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
  }
}

// 4 x 4 tile of packed block (R, C): rows 4g..4g+3, columns 4h..4h+3 (row-major in v)
template <class T>
__device__ __forceinline__ void load_tile44(const T *__restrict__ Lp, int R, int C, int g, int h,
                                            T *v) {
  const T *blk = Lp + packed_index(R, C) * NB_ * NB_ + (g * 4) * NB_ + h * 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) v[i * 4 + j] = ldg_t(blk + i * NB_ + j);
}

// column-wise slice of packed block (R, C): entries [q*16+u][c], u < 16
template <class T>
__device__ __forceinline__ void load_colslice(const T *__restrict__ Lp, int R, int C, int c, int q,
                                              T *lv) {
  const T *blk = Lp + packed_index(R, C) * NB_ * NB_ + (q * 16) * NB_ + c;
#pragma unroll
  for (int u = 0; u < 16; ++u) lv[u] = ldg_t(blk + u * NB_);
}

// this thread's 16 entries of the off-diagonal block used by row I against
// block J: FWD reads row r_f of L_IJ (contiguous), BWD column c_b of L_JI
template <class T, bool FWD>
__device__ __forceinline__ void load_block(const T *__restrict__ Lp, int I, int J, int r_f, int q_f,
                                           int c_b, int q_b, T *lv) {
  if (FWD) {
    ld16(Lp + packed_index(I, J) * NB_ * NB_ + r_f * NB_ + q_f * 16, lv);
  } else {
    const T *blk = Lp + packed_index(J, I) * NB_ * NB_ + (q_b * 16) * NB_ + c_b;
#pragma unroll
    for (int u = 0; u < 16; ++u) lv[u] = ldg_t(blk + u * NB_);
  }
}

// Block rows complete strictly in dependency order (row I needs row I-1), so
// one counter `progress` (rows finished, counted from the start for FWD and
// from the end for BWD) tells every CTA which results are ready.  A CTA reads
// it once, consumes every ready block without further synchronisation, and
// waits only for its last dependency; CTAs far behind the front poll slowly
// so the counter's cache line is not flooded.
//
// The chain step is a single 64x64 product: with the diagonal inverse
// applied ahead of time,
//   FWD  z_I = Linv_I (b_I - sum_{J<I-1} L_IJ z_J)  -  M_I z_{I-1},
//        M_I = Linv_I L_{I,I-1}
//   BWD  x_I = Linv_I^T (y_I - sum_{J>I+1} L_JI^T x_J)  -  N_I^T-form x_{I+1},
//        stored as C_I = L_{I+1,I} Linv_I so that x_I[c] -= sum_r C_I[r][c] x_{I+1}[r]
// (M_I and C_I are formed at factor time).  prog[0] = ticket, prog[1] = progress.
template <class T, bool FWD>
__global__ void __launch_bounds__(256)
k_trsv(const T *__restrict__ Lp, const T *__restrict__ Linv, const T *__restrict__ Lchain,
       const void *__restrict__ rhs, int rhs_kind, T *__restrict__ out, int nrows, int NBw,
       int *prog, int *err, int *abort_flag) {
  typedef DS<T> S;
  __shared__ T sv[NB_];
  __shared__ T sw[NB_];
  __shared__ T sred[4][NB_];
  __shared__ T spart[16][NB_ + 1];
  __shared__ int sI, sP, sbail;
  const int tid = threadIdx.x;
  // FWD: row r, column quarter q (the four quarters of a row are adjacent lanes)
  // BWD: column c, row quarter q (q = pair of warps)
  const int r_f = tid >> 2, q_f = tid & 3;
  const int c_b = tid & 63, q_b = tid >> 6;
  const int q = FWD ? q_f : q_b;
  for (;;) {
    if (tid == 0) { sI = atomicAdd(prog, 1); sbail = 0; }
    __syncthreads();
    const int ticket = sI;
    if (ticket >= NBw) return;
    const int I = FWD ? ticket : NBw - 1 - ticket;
    const int ndep = ticket;                 // blocks this row depends on
    const int rrow = FWD ? r_f : c_b;
    const long gi = (long)I * NB_ + rrow;
    const bool owner = FWD ? (q_f == 0) : (tid < NB_);
    T bval = S::zerov();
    if (owner && gi < nrows) bval = ld_rhs<T>(rhs, rhs_kind, gi);
    // ---- bulk: every dependency but the last.
    //   FWD: thread (row group g = tid/16, column group h = tid%16) sums rows
    //        4g..4g+3 of L_IJ over columns 4h..4h+3 (16 partials per row; each
    //        half-warp reads whole 512-byte rows)
    //   BWD: thread (column c, row quarter q): sum_u L_JI[q*16+u][c] x_J[q*16+u]
    //        (for each u a warp reads 32 consecutive elements)
    const int g_f = tid >> 4, h_f = tid & 15;
    T accs[FWD ? 4 : 1];
#pragma unroll
    for (int u = 0; u < (FWD ? 4 : 1); ++u) accs[u] = S::zerov();
    const int nbulk = ndep > 0 ? ndep - 1 : 0;
    int d = 0;
    T lv[16];
    // dependency d is block (I, d) for FWD and block (NBw-1-d, I) for BWD
    if (nbulk > 0) {
      if (FWD) load_tile44(Lp, I, 0, g_f, h_f, lv);
      else load_colslice(Lp, NBw - 1, I, c_b, q_b, lv);
    }
    while (d < nbulk) {
      if (tid == 0) {
        int p = ld_acquire(prog + 1);
        if (p <= d) {
          const unsigned long long t0 = global_ns();
          while ((p = ld_acquire(prog + 1)) <= d) {
            if (*(volatile int *)abort_flag) { sbail = 1; break; }
            if (global_ns() - t0 > WAIT_LIMIT_NS) {
              record_error(err, TW_ERR_TIMEOUT, FWD ? 1 : 2);
              atomicExch(abort_flag, 1);
              sbail = 1;
              break;
            }
            // rows finish every few microseconds; a CTA k rows behind the
            // front can lag k rows and catch up with one burst of blocks
            const int behind = ticket - p;
            __nanosleep(behind > 2 ? min(4096, 256 * (behind - 2)) : 32);
          }
        }
        sP = p;
      }
      __syncthreads();
      if (sbail) return;
      const int dend = min(sP, nbulk);
      for (; d < dend; ++d) {
        const int J = FWD ? d : NBw - 1 - d;
        // prefetch the next block (the stream does not depend on the chain)
        T nx[16];
        if (d + 1 < nbulk) {
          if (FWD) load_tile44(Lp, I, d + 1, g_f, h_f, nx);
          else load_colslice(Lp, NBw - 2 - d, I, c_b, q_b, nx);
        }
        if (FWD) {
          const T *zj = out + (long)J * NB_ + h_f * 4;
          T zc[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) zc[j] = ld_cg(zj + j);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) accs[i] = S::add(accs[i], S::mul(lv[i * 4 + j], zc[j]));
        } else {
          const T *zj = out + (long)J * NB_ + q_b * 16;
          typename S::acc a = S::zero();
#pragma unroll
          for (int u = 0; u < 16; ++u) S::mac(a, lv[u], ld_cg(zj + u));
          S::fold(accs[0], a);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) lv[u] = nx[u];
      }
      __syncthreads();   // sP is rewritten next round
    }
    // ---- v = b - bulk sum, w = Linv v (or Linv^T v): before the last dependency
    if (FWD) {
      // row r: sum its 16 column-group partials through shared memory
#pragma unroll
      for (int i = 0; i < 4; ++i) spart[h_f][g_f * 4 + i] = accs[i];
      __syncthreads();
      if (owner) {
        T s = spart[0][r_f];
#pragma unroll
        for (int h = 1; h < 16; ++h) s = S::add(s, spart[h][r_f]);
        sv[r_f] = (gi < nrows) ? S::sub(bval, s) : S::zerov();
      }
    } else {
      sred[q_b][c_b] = accs[0];
      __syncthreads();
      if (owner) {
        T s = S::add(S::add(sred[0][tid], sred[1][tid]), S::add(sred[2][tid], sred[3][tid]));
        sv[tid] = (gi < nrows) ? S::sub(bval, s) : S::zerov();
      }
    }
    __syncthreads();
    {
      // diagonal inverse entries: loaded here, after the bulk loop, to keep
      // registers free while the off-diagonal blocks stream
      T iv[16];
      if (FWD) {
        ld16(Linv + (size_t)I * NB_ * NB_ + r_f * NB_ + q_f * 16, iv);
      } else {
        const T *ib = Linv + (size_t)I * NB_ * NB_ + (q_b * 16) * NB_ + c_b;
#pragma unroll
        for (int u = 0; u < 16; ++u) iv[u] = ldg_t(ib + u * NB_);
      }
      typename S::acc a2 = S::zero();
#pragma unroll
      for (int u = 0; u < 16; ++u) S::mac(a2, iv[u], sv[q * 16 + u]);
      if (FWD) {
        T s = S::get(a2);
        s = S::add(s, S::shfl_xor(s, 1));
        s = S::add(s, S::shfl_xor(s, 2));
        if (owner) sw[r_f] = s;
      } else {
        __syncthreads();
        sred[q_b][c_b] = S::get(a2);
        __syncthreads();
        if (owner) sw[tid] = S::add(S::add(sred[0][tid], sred[1][tid]), S::add(sred[2][tid], sred[3][tid]));
      }
    }
    // ---- the last dependency: one product with the chain block
    T corr = S::zerov();
    if (ndep > 0) {
      // chain block entries: issued before the wait so they arrive during it
      T cv[16];
      if (FWD) {
        ld16(Lchain + (size_t)I * NB_ * NB_ + r_f * NB_ + q_f * 16, cv);
      } else {
        const T *cb = Lchain + (size_t)I * NB_ * NB_ + (q_b * 16) * NB_ + c_b;
#pragma unroll
        for (int u = 0; u < 16; ++u) cv[u] = ldg_t(cb + u * NB_);
      }
      if (tid == 0) {
        const unsigned long long t0 = global_ns();
        int p;
        while ((p = ld_acquire(prog + 1)) < ndep) {
          if (*(volatile int *)abort_flag) { sbail = 1; break; }
          if (global_ns() - t0 > WAIT_LIMIT_NS) {
            record_error(err, TW_ERR_TIMEOUT, FWD ? 3 : 4);
            atomicExch(abort_flag, 1);
            sbail = 1;
            break;
          }
          __nanosleep(32);
        }
      }
      __syncthreads();
      if (sbail) return;
      const int J = FWD ? I - 1 : I + 1;
      const T *zj = out + (long)J * NB_ + q * 16;
      typename S::acc a3 = S::zero();
#pragma unroll
      for (int u = 0; u < 16; ++u) S::mac(a3, cv[u], ld_cg(zj + u));
      if (FWD) {
        T s = S::get(a3);
        s = S::add(s, S::shfl_xor(s, 1));
        s = S::add(s, S::shfl_xor(s, 2));
        corr = s;
      } else {
        sred[q_b][c_b] = S::get(a3);
        __syncthreads();
        if (owner) corr = S::add(S::add(sred[0][tid], sred[1][tid]), S::add(sred[2][tid], sred[3][tid]));
      }
    } else {
      __syncthreads();
    }
    if (owner) out[gi] = (gi < nrows) ? S::sub(sw[rrow], corr) : S::zerov();
    __threadfence();
    __syncthreads();
    // rows finish in order, so the counter is `ticket` here; publish ticket + 1
    if (tid == 0) st_release(prog + 1, ticket + 1);
  }
}

// Chain blocks of the solves (formed once per factorisation):
//   M_I = Linv_I L_{I,I-1}  (I >= 1)     C_I = L_{I+1,I} Linv_I  (I <= NB-2)
template <class T>
__global__ void __launch_bounds__(256)
k_chain_blocks(const T *__restrict__ Lp, const T *__restrict__ Linv, T *__restrict__ Mf,
               T *__restrict__ Cb, int NB) {
  typedef DS<T> S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*sA)[NB_ + 1] = reinterpret_cast<T(*)[NB_ + 1]>(smem_raw);
  T(*sB)[NB_ + 1] = sA + NB_;
  const int I = blockIdx.x, tid = threadIdx.x;
  for (int which = 0; which < 2; ++which) {
    const bool fwd = which == 0;
    if (fwd ? I < 1 : I > NB - 2) continue;
    const T *Lb = fwd ? Lp + packed_index(I, I - 1) * NB_ * NB_ : Lp + packed_index(I + 1, I) * NB_ * NB_;
    const T *Iv = Linv + (size_t)I * NB_ * NB_;
    __syncthreads();
    for (int idx = tid; idx < NB_ * NB_; idx += blockDim.x) {
      const int r = idx / NB_, c = idx % NB_;
      sA[r][c] = fwd ? Iv[idx] : Lb[idx];     // left factor
      sB[r][c] = fwd ? Lb[idx] : Iv[idx];     // right factor
    }
    __syncthreads();
    T *dst = (fwd ? Mf : Cb) + (size_t)I * NB_ * NB_;
    for (int idx = tid; idx < NB_ * NB_; idx += blockDim.x) {
      const int r = idx / NB_, c = idx % NB_;
      typename S::acc a = S::zero();
      for (int k = 0; k < NB_; ++k) S::mac(a, sA[r][k], sB[k][c]);
      dst[idx] = S::get(a);
    }
  }
}

// ------------------------------------------- symmetric K x from packed lower
// r = d - K x over the leading nrows (df64); one CTA per block row, no
// synchronisation inside the sweep: lower blocks (J <= I) row-wise, upper
// blocks as transposes of the stored (J, I) blocks.
// d == nullptr: r = K x instead of d - K x
__global__ void __launch_bounds__(256)
k_residual(const dd *__restrict__ Kp, const dd *__restrict__ x, const double *__restrict__ d,
           dd *__restrict__ r, int nrows, int NBw) {
  __shared__ dd sN[NB_];
  __shared__ dd sT[4][NB_];
  const int I = blockIdx.x, tid = threadIdx.x;
  const int r_f = tid >> 2, q_f = tid & 3;     // lower blocks (J <= I)
  const int c_b = tid & 63, q_b = tid >> 6;    // transposed blocks (J > I)
  dd totN = dd_zero(), totT = dd_zero();
  for (int J = 0; J < NBw; ++J) {
    dacc a = dacc_zero();
    if (J <= I) {
      const dd *blk = Kp + packed_index(I, J) * NB_ * NB_;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int c = q_f * 16 + u;
        // diagonal block: the stored upper part is zero, use the lower entry
        const dd kv = (I == J && c > r_f) ? blk[c * NB_ + r_f] : blk[r_f * NB_ + c];
        const long gj = (long)J * NB_ + c;
        dacc_mac(a, kv, (gj < nrows) ? x[gj] : dd_zero());
      }
      dacc_fold(totN, a);
    }
    if (J > I) {
      const dd *blk = Kp + packed_index(J, I) * NB_ * NB_ + c_b;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int rr = q_b * 16 + u;
        const long gj = (long)J * NB_ + rr;
        dacc_mac(a, blk[rr * NB_], (gj < nrows) ? x[gj] : dd_zero());
      }
      dacc_fold(totT, a);
    }
  }
  dd s = totN;
  s = dd_add(s, DS<dd>::shfl_xor(s, 1));
  s = dd_add(s, DS<dd>::shfl_xor(s, 2));
  if (q_f == 0) sN[r_f] = s;
  sT[q_b][c_b] = totT;
  __syncthreads();
  if (tid < NB_) {
    dd t = dd_add(dd_add(sT[0][tid], sT[1][tid]), dd_add(sT[2][tid], sT[3][tid]));
    t = dd_add(t, sN[tid]);
    const long gi = (long)I * NB_ + tid;
    r[gi] = (gi < nrows) ? (d ? dd_sub(dd_from_double(d[gi]), t) : t) : dd_zero();
  }
}

__global__ void k_dd_to_double(const dd *__restrict__ a, double *__restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = dd_to_double(a[i]);
}
__global__ void k_double_to_dd_vec(const double *__restrict__ a, dd *__restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = dd_from_double(a[i]);
}

// r[i] = d[i] - a[i] - sigma z[i] for i < n (time-major data vectors, the
// leading n = Nd Nt' rows; the rest of r is left alone)
__global__ void k_sample_rhs(const double *__restrict__ d, const double *__restrict__ a,
                             const double *__restrict__ z, double sigma, double *__restrict__ r, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = d[i] - a[i] - sigma * z[i];
}
// s[i] += x[i] (x double-float) for i < n
__global__ void k_add_dd(double *__restrict__ s, const dd *__restrict__ x, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) s[i] += dd_to_double(x[i]);
}

// x += delta (float) ; rows < nrows
__global__ void k_axpy_dd_f(dd *__restrict__ x, const float *__restrict__ delta, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { dd d; d.hi = delta[i]; d.lo = 0.f; x[i] = dd_add(x[i], d); }
}
// float -> dd copy
__global__ void k_f_to_dd(const float *__restrict__ a, dd *__restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { b[i].hi = a[i]; b[i].lo = 0.f; }
}
// sum of squares (double) of dd (kind 1) or double (kind 0) vector, atomically added
__global__ void k_sumsq(const void *__restrict__ v, int kind, int n, double *out) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double x;
    if (kind == 0) x = reinterpret_cast<const double *>(v)[i];
    else { const dd t = reinterpret_cast<const dd *>(v)[i]; x = (double)t.hi + (double)t.lo; }
    s += x * x;
  }
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

template <class KER> void smem_attr(KER k, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ======================================================================= host
cudaError_t launch_K_from_P(double *K, long ldk, int Nd, int Nt, int n, int n_pad, double sigma2,
                            cudaStream_t s) {
  const long total = (long)Nt * Nd * Nd;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_prefix_diag<<<(unsigned)blocks, 256, 0, s>>>(K, ldk, Nd, Nt);
  count_launches(1);
  k_diag_set<<<(n_pad + 255) / 256, 256, 0, s>>>(K, ldk, n, n_pad, sigma2);
  count_launches(1);
  return cudaGetLastError();
}

// Right-looking blocked Cholesky, 64-wide panels, rank-64 trailing updates
// as SIMT products.
template <class T>
cudaError_t cholesky_t(T *K, long ldk, int NB, T *inv, int *err, cudaStream_t s) {
  const size_t sm_potrf = 2 * NB_ * (NB_ + 1) * sizeof(T);
  const size_t sm_trsm = 2 * NB_ * (NB_ + 1) * sizeof(T);
  smem_attr(k_potrf_diag<T>, sm_potrf);
  smem_attr(k_trsm_panel<T>, sm_trsm);
  for (int J = 0; J < NB; ++J) {
    T *diag = K + (long)J * NB_ * ldk + (long)J * NB_;
    k_potrf_diag<T><<<1, 256, sm_potrf, s>>>(K, ldk, J, inv + (size_t)J * NB_ * NB_, err);
    count_launches(1);
    const int nt = NB - J - 1;
    if (nt > 0) {
      k_trsm_panel<T><<<nt, 64, sm_trsm, s>>>(K, ldk, J);
      count_launches(1);
      const T *panel = diag + (long)NB_ * ldk;               // rows (J+1)*64.., cols J*64..
      T *trail = diag + (long)NB_ * ldk + NB_;
      k_gemm_nt<T><<<dim3(nt, nt), 256, 0, s>>>(panel, ldk, nt * NB_, panel, ldk, nt * NB_, NB_,
                                                trail, ldk, 1, 1);
      count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_cholesky_f(float *K, long ldk, int NB, float *inv, int *err, cudaStream_t s) {
  return cholesky_t<float>(K, ldk, NB, inv, err, s);
}

// FP64 with the trailing updates on the tensor cores: super-steps of SW
// block columns.  Within a super-step each column first takes the deferred
// updates of the super-step's earlier columns (FP64 SIMT, k <= 64 (SW-1)),
// then its diagonal block and panel; the trailing matrix then takes one
// rank-64 SW update (exact products, gemm_syrk.cu), so the update's FP64
// read-modify-write of K is paid once per SW columns.
constexpr int CHOL_SW = 4;
int cholesky_tc_width() { return CHOL_SW; }

cudaError_t launch_cholesky_d(double *K, long ldk, int NB, double *inv, int *err, uint8_t *ws,
                              size_t ws_bytes, int *eg, cudaStream_t s) {
  if (!ws) return cholesky_t<double>(K, ldk, NB, inv, err, s);
  const size_t sm_potrf = 2 * NB_ * (NB_ + 1) * sizeof(double);
  const size_t sm_trsm = 2 * NB_ * (NB_ + 1) * sizeof(double);
  smem_attr(k_potrf_diag<double>, sm_potrf);
  smem_attr(k_trsm_panel<double>, sm_trsm);
  for (int J0 = 0; J0 < NB; J0 += CHOL_SW) {
    const int w = std::min(CHOL_SW, NB - J0);
    for (int jj = 0; jj < w; ++jj) {
      const int J = J0 + jj, nrow = NB - J;
      double *colJ = K + (long)J * NB_ * ldk + (long)J * NB_;
      if (jj > 0) {
        // block column J, rows J..: minus L(rows, J0..J-1) L(J, J0..J-1)^T
        const double *A = K + (long)J * NB_ * ldk + (long)J0 * NB_;
        k_gemm_nt<double><<<dim3(1, nrow), 256, 0, s>>>(A, ldk, nrow * NB_, A, ldk, NB_, jj * NB_, colJ,
                                                        ldk, 0, 1);
        count_launches(1);
      }
      k_potrf_diag<double><<<1, 256, sm_potrf, s>>>(K, ldk, J, inv + (size_t)J * NB_ * NB_, err);
      count_launches(1);
      if (nrow > 1) {
        k_trsm_panel<double><<<nrow - 1, 64, sm_trsm, s>>>(K, ldk, J);
        count_launches(1);
      }
    }
    const int m = (NB - J0 - w) * NB_;
    if (m > 0) {
      const double *A = K + (long)(J0 + w) * NB_ * ldk + (long)J0 * NB_;
      double *C = K + (long)(J0 + w) * NB_ * ldk + (long)(J0 + w) * NB_;
      cudaError_t e = launch_syrk_update_d(A, ldk, w * NB_, C, ldk, m, ws, ws_bytes, eg, err, s);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t launch_pack_d(const double *K, long ldk, double *P, int NB, cudaStream_t s) {
  k_pack<double><<<152 * 8, 256, 0, s>>>(K, ldk, P, NB);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_pack_d2dd(const double *K, long ldk, dd *P, int NB, cudaStream_t s) {
  k_pack_d2dd<<<152 * 8, 256, 0, s>>>(K, ldk, P, NB);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_double_to_dd(const double *a, dd *b, size_t n, cudaStream_t s) {
  k_double_to_dd<<<152 * 16, 256, 0, s>>>(a, b, n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_f(const float *K, long ldk, float *P, int NB, cudaStream_t s) {
  k_pack<float><<<152 * 8, 256, 0, s>>>(K, ldk, P, NB);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_lower_to_float(const double *K, float *K32, long ld, int NB, cudaStream_t s) {
  k_lower_to_float<<<dim3(NB, NB), 256, 0, s>>>(K, K32, ld, NB);
  count_launches(1);
  return cudaGetLastError();
}

static int trsv_grid(int NBw) { return NBw < 152 * 4 ? NBw : 152 * 4; }

cudaError_t launch_trsv_f(const float *Lp, const float *Linv, const float *Lchain,
                          const void *rhs, int rhs_kind, float *out, int nrows, int NBw, int *prog,
                          bool fwd, int *err, int *abort_flag, cudaStream_t s) {
  if (NBw <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(prog, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (fwd)
    k_trsv<float, true><<<trsv_grid(NBw), 256, 0, s>>>(Lp, Linv, Lchain, rhs, rhs_kind, out,
                                                               nrows, NBw, prog, err, abort_flag);
  else
    k_trsv<float, false><<<trsv_grid(NBw), 256, 0, s>>>(Lp, Linv, Lchain, rhs, rhs_kind, out,
                                                                nrows, NBw, prog, err, abort_flag);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chain_blocks_d(const double *Lp, const double *Linv, double *Mf, double *Cb,
                                  int NB, cudaStream_t s) {
  const size_t sm = 2 * NB_ * (NB_ + 1) * sizeof(double);
  smem_attr(k_chain_blocks<double>, sm);
  k_chain_blocks<double><<<NB, 256, sm, s>>>(Lp, Linv, Mf, Cb, NB);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_chain_blocks_f(const float *Lp, const float *Linv, float *Mf, float *Cb, int NB,
                                  cudaStream_t s) {
  const size_t sm = 2 * NB_ * (NB_ + 1) * sizeof(float);
  smem_attr(k_chain_blocks<float>, sm);
  k_chain_blocks<float><<<NB, 256, sm, s>>>(Lp, Linv, Mf, Cb, NB);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_residual(const dd *Kp, const dd *x, const double *d, dd *r, int nrows, int NBw,
                            cudaStream_t s) {
  if (NBw <= 0) return cudaSuccess;
  k_residual<<<NBw, 256, 0, s>>>(Kp, x, d, r, nrows, NBw);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_dd_to_double(const dd *a, double *b, int n, cudaStream_t s) {
  k_dd_to_double<<<(n + 255) / 256, 256, 0, s>>>(a, b, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_double_to_dd_vec(const double *a, dd *b, int n, cudaStream_t s) {
  k_double_to_dd_vec<<<(n + 255) / 256, 256, 0, s>>>(a, b, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_sample_rhs(const double *d, const double *a, const double *z, double sigma,
                              double *r, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_sample_rhs<<<(n + 255) / 256, 256, 0, s>>>(d, a, z, sigma, r, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_add_dd(double *sv, const dd *x, long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_add_dd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sv, x, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_axpy_dd_f(dd *x, const float *delta, int n, cudaStream_t s) {
  k_axpy_dd_f<<<(n + 255) / 256, 256, 0, s>>>(x, delta, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_f_to_dd(const float *a, dd *b, int n, cudaStream_t s) {
  k_f_to_dd<<<(n + 255) / 256, 256, 0, s>>>(a, b, n);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t launch_sumsq(const void *v, int kind, int n, double *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  int blocks = (n + 255) / 256;
  if (blocks > 152 * 4) blocks = 152 * 4;
  if (blocks < 1) blocks = 1;
  k_sumsq<<<blocks, 256, 0, s>>>(v, kind, n, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tw
