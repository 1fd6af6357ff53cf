// trsv64.cu -- the FP64 triangular solves of one right-hand side.
//
// Online, y = K'^-1 d' is a forward sweep L z = d and a backward sweep
// L^T y = z with K's Cholesky factor (Phase 4; windows use its leading
// rows).  The sweeps are bound by FP64 FMA throughput (n^2/2 DFMA each) and by
// the row-to-row dependency chain.  This file reformulates them so that
// neither the chain nor the load balance limits the sweep:
//
//  * Block-scaled factor (formed once per factorisation):
//      forward   z_I = Linv_I b_I - sum_{J<I} Lf_IJ z_J,      Lf_IJ = Linv_I L_IJ
//      backward  x_I = Linv_I^T y_I - sum_{J>I} Lb_JI^T x_J,  Lb_JI = L_JI Linv_I
//    (Linv_I the inverse of the diagonal block), so no product with Linv
//    waits on the chain.
//  * Chain CTA (block 0) applies the two most recent dependencies,
//      z_u = w_u - A1_u z_{u-1} - A2_u z_{u-2},
//    keeping z_{u-1}, z_{u-2} in shared memory and the next rows' blocks
//    A1, A2 in a four-slot shared ring filled by asynchronous copies.
//  * Workers (blocks >= 1) take tasks in row order: task (u, k) sums the
//    dependencies d in [16k, min(16k+16, u-2)) of row u (plus Linv_I b_I for
//    k = 0) into a partial vector; the task that completes a row adds its
//    partials in chunk order (deterministic) and hands w_u to the chain CTA.
//    Long rows are thus spread over many CTAs.
// u is the row's position in dependency order (forward: I = u; backward:
// I = NBw-1-u) and d a dependency's position (forward J = d; backward
// J = NBw-1-d).  All waits are bounded (2 s -> TW_ERR_TIMEOUT, abort flag).
#include <algorithm>
#include <vector>

#include "../../include/tw.h"
#include "dense_api.h"
#include "kernels.h"

namespace tw {

namespace {

constexpr int CH = 16;                      // dependencies per worker task
constexpr unsigned long long WAIT_NS = 2000000000ull;
constexpr int BLK = NB_ * NB_;

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int acq(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void rel(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void err_note(int *err, int code, int info) {
  if (atomicCAS(err, 0, code) == 0) err[1] = info;
}

// number of worker tasks of row u
__host__ __device__ __forceinline__ int row_tasks(int u) {
  const int nd = u > 2 ? u - 2 : 0;
  return nd > 0 ? (nd + CH - 1) / CH : 1;
}

// ------------------------------------------------------------------ chain CTA
// The CTA owns its SM (the kernel's 128 KB of dynamic shared memory leave
// room for one CTA per SM), so its two 64x64 products per row run at the
// SM's full FP64 rate; the next rows' blocks stream into a four-slot ring.
__device__ __forceinline__ void cp16(void *dst, const void *src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
}

template <bool FWD>
__device__ void chain_role(const double *__restrict__ band1, const double *__restrict__ band2,
                           const double *__restrict__ Lb, const double *__restrict__ wbuf,
                           const int *wflag, double *__restrict__ out, int nrows, int NBw,
                           int *progress, int *err, int *abort_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *ring = reinterpret_cast<double *>(smem_raw);    // [4][64*64]
  __shared__ double zh[2][NB_];                          // z_{u-1}, z_{u-2} (by parity)
  __shared__ double red[4][NB_];
  __shared__ int bail;
  const int tid = threadIdx.x, c = tid & 63, q = tid >> 6;
  // block A_j of row v: FWD transposed band j at row I; BWD Lb block (I+j, I)
  auto blockp = [&](int v, int j) -> const double * {
    const int I = FWD ? v : NBw - 1 - v;
    if (FWD) return (j == 1 ? band1 : band2) + (size_t)I * BLK;
    return Lb + packed_index(I + j, I) * BLK;
  };
  auto stage_row = [&](int v) {   // one commit group per row, empty past the end
    if (v < NBw) {
      for (int j = 1; j <= 2; ++j) {
        if (v < j) continue;
        double *dst = ring + ((2 * v + j - 1) & 3) * BLK;
        const double *src = blockp(v, j);
        for (int i = tid; i < BLK / 2; i += blockDim.x) cp16(dst + 2 * i, src + 2 * i);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (tid == 0) bail = 0;
  stage_row(0);
  stage_row(1);
  for (int u = 0; u < NBw; ++u) {
    const int I = FWD ? u : NBw - 1 - u;
    if (tid == 0) {
      const unsigned long long t0 = gtime();
      while (acq(wflag + I) == 0) {
        if (*(volatile int *)abort_flag) { bail = 1; break; }
        if (gtime() - t0 > WAIT_NS) {
          err_note(err, TW_ERR_TIMEOUT, FWD ? 11 : 12);
          atomicExch(abort_flag, 1);
          bail = 1;
          break;
        }
      }
    }
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // row u's blocks are in
    __syncthreads();
    if (bail) { asm volatile("cp.async.wait_all;" ::: "memory"); return; }
    const long gi = (long)I * NB_ + c;
    const double w = (q == 0) ? __ldcg(wbuf + gi) : 0.0;   // in flight during the product
    double a = 0.0;
#pragma unroll
    for (int j = 1; j <= 2; ++j) {
      if (u < j) continue;
      const double *A = ring + ((2 * u + j - 1) & 3) * BLK;
      const double *zp = zh[(u - j) & 1];
#pragma unroll
      for (int k = q * 16; k < q * 16 + 16; ++k) a = fma(A[k * NB_ + c], zp[k], a);
    }
    red[q][c] = a;
    __syncthreads();           // partials in; row u's slots and z_{u-2} consumed
    stage_row(u + 2);          // into row u's slots
    if (q == 0) {
      double z = w - ((red[0][c] + red[1][c]) + (red[2][c] + red[3][c]));
      z = gi < nrows ? z : 0.0;
      out[gi] = z;
      zh[u & 1][c] = z;        // overwrites z_{u-2}
    }
    // the barrier orders every thread's stores before thread 0's release,
    // which is cumulative: one release publishes the row
    __syncthreads();
    if (tid == 0) rel(progress, u + 1);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// ------------------------------------------------------------------ workers
__device__ __forceinline__ double ld_b(const void *rhs, int kind, long i) {
  if (kind == 0) return __ldcg(reinterpret_cast<const double *>(rhs) + i);
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(rhs) + i);
  return (double)v.x + (double)v.y;
}

template <bool FWD>
__device__ void worker_role(const double *__restrict__ Lx, const double *__restrict__ Linv,
                            const void *__restrict__ rhs, int rhs_kind, const double *__restrict__ zout,
                            const int2 *__restrict__ tasks, int ntasks, double *__restrict__ part,
                            int maxk, int *cnt, double *__restrict__ wbuf, int *wflag, int nrows,
                            int NBw, int *prog, int *err, int *abort_flag) {
  __shared__ double sv[NB_];
  __shared__ double spart[16][NB_ + 1];
  __shared__ double sred[4][NB_];
  __shared__ int sT, sP, sbail, slast;
  const int tid = threadIdx.x;
  const int r_f = tid >> 2, q_f = tid & 3;        // FWD row r, column quarter
  const int c_b = tid & 63, q_b = tid >> 6;       // BWD column c, row quarter
  const int g_f = tid >> 4, h_f = tid & 15;       // FWD bulk 4x4 tiles
  int *progress = prog + 1;
  for (;;) {
    __syncthreads();
    if (tid == 0) { sT = atomicAdd(prog, 1); sbail = 0; }
    __syncthreads();
    const int t = sT;
    if (t >= ntasks) return;
    const int u = tasks[t].x, k = tasks[t].y;
    const int I = FWD ? u : NBw - 1 - u;
    const int rrow = FWD ? r_f : c_b;
    const long gi = (long)I * NB_ + rrow;
    const bool owner = FWD ? (q_f == 0) : (tid < NB_);
    // ---- this task's dependencies: d in [d0, d1)
    const int nd = u > 2 ? u - 2 : 0;
    const int d0 = k * CH, d1 = min(nd, d0 + CH);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    auto dblock = [&](int d) -> const double * {
      const int J = FWD ? d : NBw - 1 - d;
      return Lx + (FWD ? packed_index(I, J) : packed_index(J, I)) * BLK;
    };
    double lv[16];
    auto load = [&](int d, double *v) {
      const double *blk = dblock(d);
      if (FWD) {
        const double *p = blk + (g_f * 4) * NB_ + h_f * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) v[i * 4 + j] = __ldg(p + i * NB_ + j);
      } else {
        const double *p = blk + (q_b * 16) * NB_ + c_b;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __ldg(p + i * NB_);
      }
    };
    int d = d0;
    if (d < d1) load(d, lv);
    while (d < d1) {
      if (tid == 0) {
        int p = acq(progress);
        if (p <= d) {
          const unsigned long long t0 = gtime();
          while ((p = acq(progress)) <= d) {
            if (*(volatile int *)abort_flag) { sbail = 1; break; }
            if (gtime() - t0 > WAIT_NS) {
              err_note(err, TW_ERR_TIMEOUT, FWD ? 13 : 14);
              atomicExch(abort_flag, 1);
              sbail = 1;
              break;
            }
            const int behind = d - p;
            __nanosleep(behind > 2 ? min(4096, 256 * (behind - 2)) : 32);
          }
        }
        sP = p;
      }
      __syncthreads();
      if (sbail) return;
      const int dend = min(sP, d1);
      for (; d < dend; ++d) {
        const int J = FWD ? d : NBw - 1 - d;
        double nx[16];
        if (d + 1 < d1) load(d + 1, nx);
        if (FWD) {
          const double *zj = zout + (long)J * NB_ + h_f * 4;
          double zc[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) zc[j] = __ldcg(zj + j);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i] = fma(lv[i * 4 + j], zc[j], acc[i]);
        } else {
          const double *zj = zout + (long)J * NB_ + q_b * 16;
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[0] = fma(lv[i], __ldcg(zj + i), acc[0]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) lv[i] = nx[i];
      }
      __syncthreads();
    }
    // ---- chunk sum per row (64 values)
    double csum = 0.0;
    if (FWD) {
#pragma unroll
      for (int i = 0; i < 4; ++i) spart[h_f][g_f * 4 + i] = acc[i];
      __syncthreads();
      if (owner) {
        double s = spart[0][r_f];
#pragma unroll
        for (int h = 1; h < 16; ++h) s += spart[h][r_f];
        csum = s;
      }
    } else {
      sred[q_b][c_b] = acc[0];
      __syncthreads();
      if (owner) csum = (sred[0][tid] + sred[1][tid]) + (sred[2][tid] + sred[3][tid]);
    }
    // ---- k = 0 also carries Linv_I b_I (FWD) / Linv_I^T y_I (BWD)
    double res = -csum;
    if (k == 0) {
      if (owner) sv[rrow] = gi < nrows ? ld_b(rhs, rhs_kind, gi) : 0.0;
      __syncthreads();
      const double *iv = Linv + (size_t)I * BLK;
      double a2 = 0.0;
      if (FWD) {
        const double *p = iv + r_f * NB_ + q_f * 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) a2 = fma(__ldg(p + i), sv[q_f * 16 + i], a2);
        a2 += __shfl_xor_sync(0xffffffffu, a2, 1);
        a2 += __shfl_xor_sync(0xffffffffu, a2, 2);
        if (owner) res += a2;
      } else {
        const double *p = iv + (q_b * 16) * NB_ + c_b;
#pragma unroll
        for (int i = 0; i < 16; ++i) a2 = fma(__ldg(p + i * NB_), sv[q_b * 16 + i], a2);
        __syncthreads();
        sred[q_b][c_b] = a2;
        __syncthreads();
        if (owner) res += (sred[0][tid] + sred[1][tid]) + (sred[2][tid] + sred[3][tid]);
      }
    }
    const int nk = row_tasks(u);
    double *pu = part + ((size_t)u * maxk) * NB_;
    if (owner) pu[(size_t)k * NB_ + rrow] = res;
    __syncthreads();
    if (tid == 0) {
      // release the partial (fence after the barrier, then the count), and
      // acquire the other tasks' partials if this one completes the row
      __threadfence();
      const int done = atomicAdd(cnt + u, 1);
      slast = (done == nk - 1);
      __threadfence();
    }
    __syncthreads();
    if (!slast) continue;
    // ---- last task of row u: add the partials in chunk order, hand off w_u
    if (owner) {
      double w = __ldcg(pu + rrow);
      for (int kk = 1; kk < nk; ++kk) w += __ldcg(pu + (size_t)kk * NB_ + rrow);
      wbuf[gi] = gi < nrows ? w : 0.0;
    }
    __syncthreads();
    if (tid == 0) rel(wflag + I, 1);   // cumulative release of the CTA's stores
  }
}

template <bool FWD>
__global__ void __launch_bounds__(256)
k_trsv64(const double *__restrict__ Lx, const double *__restrict__ Linv,
         const double *__restrict__ band1, const double *__restrict__ band2,
         const void *__restrict__ rhs, int rhs_kind, double *__restrict__ out, int nrows, int NBw,
         const int2 *__restrict__ tasks, int ntasks, double *__restrict__ part, int maxk, int *cnt,
         double *__restrict__ wbuf, int *wflag, int *prog, int *err, int *abort_flag) {
  if (blockIdx.x == 0)
    chain_role<FWD>(band1, band2, Lx, wbuf, wflag, out, nrows, NBw, prog + 1, err, abort_flag);
  else
    worker_role<FWD>(Lx, Linv, rhs, rhs_kind, out, tasks, ntasks, part, maxk, cnt, wbuf, wflag,
                     nrows, NBw, prog, err, abort_flag);
}

// ------------------------------------------------------------- set-up kernels
// per packed block (I, J), J < I:  Lf = Linv_I L_IJ,  Lb = L_IJ Linv_J
__global__ void __launch_bounds__(256)
k_scale_blocks(const double *__restrict__ Lp, const double *__restrict__ Linv,
               double *__restrict__ Lf, double *__restrict__ Lb, int NB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double(*sL)[NB_ + 1] = reinterpret_cast<double(*)[NB_ + 1]>(smem_raw);
  double(*sA)[NB_ + 1] = sL + NB_;
  double(*sB)[NB_ + 1] = sA + NB_;
  // block index -> (I, J): I(I+1)/2 + J = blockIdx.x
  const long b = blockIdx.x;
  int I = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) / 2.0);
  while ((long)I * (I + 1) / 2 > b) --I;
  while ((long)(I + 1) * (I + 2) / 2 <= b) ++I;
  const int J = (int)(b - (long)I * (I + 1) / 2);
  if (J >= I) return;                      // diagonal blocks are not used
  const double *L = Lp + (size_t)b * BLK;
  const double *Ai = Linv + (size_t)I * BLK, *Bj = Linv + (size_t)J * BLK;
  for (int i = threadIdx.x; i < BLK; i += blockDim.x) {
    sL[i / NB_][i % NB_] = L[i];
    sA[i / NB_][i % NB_] = Ai[i];
    sB[i / NB_][i % NB_] = Bj[i];
  }
  __syncthreads();
  const int r = threadIdx.x >> 2, c0 = threadIdx.x & 3;
#pragma unroll 1
  for (int j = 0; j < 16; ++j) {
    const int c = c0 + 4 * j;
    double f = 0.0, g = 0.0;
#pragma unroll 8
    for (int kk = 0; kk < NB_; ++kk) {
      f = fma(sA[r][kk], sL[kk][c], f);      // (Linv_I L_IJ)[r][c]
      g = fma(sL[r][kk], sB[kk][c], g);      // (L_IJ Linv_J)[r][c]
    }
    Lf[(size_t)b * BLK + r * NB_ + c] = f;
    Lb[(size_t)b * BLK + r * NB_ + c] = g;
  }
}

// FWD chain blocks, transposed: band_j[I] = Lf_{I,I-j}^T (I >= j)
__global__ void k_bands_t(const double *__restrict__ Lf, double *__restrict__ band1,
                          double *__restrict__ band2, int NB) {
  __shared__ double t[NB_][NB_ + 1];
  const int I = blockIdx.x, j = blockIdx.y + 1;
  if (I < j) return;
  const double *src = Lf + packed_index(I, I - j) * BLK;
  for (int i = threadIdx.x; i < BLK; i += blockDim.x) t[i / NB_][i % NB_] = src[i];
  __syncthreads();
  double *dst = (j == 1 ? band1 : band2) + (size_t)I * BLK;
  for (int i = threadIdx.x; i < BLK; i += blockDim.x) dst[i] = t[i % NB_][i / NB_];
}

}  // namespace

// ------------------------------------------------------------------ host side
int trsv64_max_tasks_per_row(int NB) { return row_tasks(std::max(NB - 1, 0)); }

void trsv64_task_table(int NB, std::vector<int> &tab, std::vector<int> &prefix) {
  tab.clear();
  prefix.assign(NB + 1, 0);
  for (int u = 0; u < NB; ++u) {
    prefix[u] = (int)(tab.size() / 2);
    for (int k = 0; k < row_tasks(u); ++k) { tab.push_back(u); tab.push_back(k); }
  }
  prefix[NB] = (int)(tab.size() / 2);
}

cudaError_t launch_trsv64_setup(const double *Lp, const double *Linv, double *Lf, double *Lb,
                                double *band1, double *band2, int NB, cudaStream_t s) {
  if (NB <= 0) return cudaSuccess;
  const size_t sm = 3 * NB_ * (NB_ + 1) * sizeof(double);
  cudaFuncSetAttribute(k_scale_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const long nblk = (long)NB * (NB + 1) / 2;
  k_scale_blocks<<<(unsigned)nblk, 256, sm, s>>>(Lp, Linv, Lf, Lb, NB);
  count_launches(1);
  k_bands_t<<<dim3(NB, 2), 256, 0, s>>>(Lf, band1, band2, NB);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_trsv64(const Trsv64Args &a, bool fwd, cudaStream_t s) {
  if (a.NBw <= 0) return cudaSuccess;
  const size_t sm = 4 * (size_t)BLK * sizeof(double);
  static int resident[64][2] = {{0}};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int &res = resident[dev][fwd ? 1 : 0];
  if (!res) {
    auto ker = fwd ? k_trsv64<true> : k_trsv64<false>;
    cudaFuncSetAttribute(ker, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0, nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ker, 256, sm);
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    res = std::max(2, per_sm * nsm);
  }
  cudaError_t e = cudaMemsetAsync(a.prog, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.wflag, 0, a.NBw * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.cnt, 0, a.NBw * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = std::min(a.ntasks + 1, res);
  if (fwd)
    k_trsv64<true><<<grid, 256, sm, s>>>(a.Lf, a.Linv, a.band1, a.band2, a.rhs, a.rhs_kind, a.out,
                                         a.nrows, a.NBw, a.tasks, a.ntasks, a.part, a.maxk, a.cnt,
                                         a.wbuf, a.wflag, a.prog, a.err, a.abort_flag);
  else
    k_trsv64<false><<<grid, 256, sm, s>>>(a.Lb, a.Linv, nullptr, nullptr, a.rhs, a.rhs_kind, a.out,
                                          a.nrows, a.NBw, a.tasks, a.ntasks, a.part, a.maxk, a.cnt,
                                          a.wbuf, a.wflag, a.prog, a.err, a.abort_flag);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tw
