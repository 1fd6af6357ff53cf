// trsv64.cu -- the FP64-class triangular solves of one right-hand side.
//
// Online, y = K'^-1 d' is a forward sweep L z = d and a backward sweep
// L^T y = z with K's Cholesky factor (Phase 4; windows use its leading
// rows).  A sweep reads the n^2/2 entries of the factor once and does one
// multiply-add with each.  GB300's FP64 pipe issues about 1.6 DFMA per clock
// per SM, which would hold a sweep near three times its HBM time, so the
// products run in double-float arithmetic on the FP32 pipes: the scaled
// factor is stored as float pairs (8 bytes an entry, like a double; relative
// representation error <= 2^-48), every product is an exact FMA two-product
// added with TwoSum into a renormalised float-pair sum, and a sweep streams
// the factor at HBM speed.  The diagonal-block inverses stay FP64.
//
//  * Block-scaled factor (formed once per factorisation, in FP64):
//      forward   z_I = Linv_I b_I - sum_{J<I} Lf_IJ z_J,      Lf_IJ = Linv_I L_IJ
//      backward  x_I = Linv_I^T y_I - sum_{J>I} Lb_JI^T x_J,  Lb_JI = L_JI Linv_I
//    (Linv_I the inverse of the diagonal block), so no product with Linv
//    waits on the chain.
//  * Chain CTA (block 0) applies the DCH = 2 most recent dependencies,
//      z_u = w_u - A1_u z_{u-1} - A2_u z_{u-2},
//    keeping z_{u-1}, z_{u-2} in shared memory (as packed operands) and the
//    next rows' blocks in a shared ring filled by bulk copies.
//  * Workers (blocks >= 1) take tasks in row order: task (u, k) sums the
//    dependencies d in [16k, min(16k+16, u-2)) of row u (plus Linv_I b_I for
//    k = 0) into a partial vector, streaming the task's blocks through the
//    same six-slot ring five blocks ahead of the products.  A row's last
//    task adds the other tasks' partials in chunk order (deterministic) and
//    hands w_u to the chain CTA.  Long rows are thus spread over many CTAs,
//    and a row's hand-offs span DCH + 1 rows of the chain.
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
constexpr int DCH = 2;                      // dependencies the chain CTA applies (u-1 .. u-DCH)
constexpr int RING = 6;                     // shared slots of 64x64 float-pair blocks (192 KB)
static_assert(2 * DCH <= RING, "the chain CTA double-buffers its DCH blocks in the ring");

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
__device__ __forceinline__ void err_note(int *err, int code, int info) {
  if (atomicCAS(err, 0, code) == 0) err[1] = info;
}
// float pairs written by other CTAs of this launch: read through L2
__device__ __forceinline__ dd ld_dd_cg(const dd *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  dd r; r.hi = v.x; r.lo = v.y; return r;
}
__device__ __forceinline__ void st_dd(dd *p, dd v) {
  *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo);
}

// number of worker tasks of row u
__host__ __device__ __forceinline__ int row_tasks(int u) {
  const int nd = u > DCH ? u - DCH : 0;
  return nd > 0 ? (nd + CH - 1) / CH : 1;
}

// ---- bulk copies of whole 32 KB blocks into ring slots, one mbarrier a slot
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, unsigned parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\t"
               "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.b32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// true once the phase with this parity has completed, false after WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint32_t bar, unsigned parity) {
  unsigned long long t0 = 0;
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      const unsigned long long t = gtime();
      if (t0 == 0) t0 = t;
      else if (t - t0 > WAIT_NS) return false;
    }
  }
}
// block src -> slot (one thread): the copy engine moves the 32 KB and
// completes the slot's phase when the bytes have landed
__device__ __forceinline__ void stage_block(uint32_t slot, uint32_t bar, const dd *src) {
  constexpr unsigned BYTES = BLK * sizeof(dd);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(BYTES) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(slot), "l"(src), "r"(BYTES), "r"(bar) : "memory");
}

// ---- hand-offs without flags: w_u (from the row's last task to the chain)
// and z_u (from the chain to the workers) are stored as 64-bit float pairs
// into buffers that the launcher fills with W_EMPTY, and the reader polls the
// entries it needs.  Arithmetic never yields W_EMPTY (both halves 0xffffffff,
// a NaN no FP32 operation produces); a stored value equal to it is replaced
// by the canonical NaN.
constexpr unsigned long long W_EMPTY = ~0ull;
__device__ __forceinline__ unsigned long long dd_bits(dd v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.hi), "f"(v.lo));
  return r;
}
__device__ __forceinline__ dd bits_dd(unsigned long long b) {
  dd r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.hi), "=f"(r.lo) : "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const dd *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_flag(dd *p, dd v) {
  unsigned long long b = dd_bits(v);
  if (b == W_EMPTY) b = 0x7fffffff7fffffffull;
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}

// ------------------------------------------------------------------ chain CTA
// The CTA owns its SM (the kernel's 192 KB of dynamic shared memory leave
// room for one CTA per SM); the next row's blocks stream into the ring while
// the current row's DCH 64x64 products run.
template <bool FWD>
__device__ void chain_role(const dd *__restrict__ bands, int NBb, const dd *__restrict__ wbuf,
                           double *__restrict__ out, dd *__restrict__ outx, int nrows, int NBw,
                           int *progress, int *err, int *abort_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd *ring = reinterpret_cast<dd *>(smem_raw);          // [RING][64*64]
  // z_v (at v mod DCH) as the packed operands of the products: (hi, hi),
  // (-hi, -hi), (lo, lo)
  struct ZP { f2 hh, nn, ll, pad; };
  __shared__ __align__(16) ZP zp[DCH][NB_];
  __shared__ dd red[8][NB_];
  __shared__ __align__(8) unsigned long long sbar[RING];
  __shared__ int bail;
  const int tid = threadIdx.x, c = tid & 63, q = tid >> 6;
  // products: columns 2 c2, 2 c2 + 1 (one FP32 lane each), terms 8 kq .. 8 kq + 7
  const int c2 = tid & 31, kq = tid >> 5;
  // block A_j of row v (split planes): FWD Lf_{I,I-j}^T, BWD Lb_{I+j,I}
  auto blockp = [&](int v, int j) -> const dd * {
    const int I = FWD ? v : NBw - 1 - v;
    return bands + ((size_t)(j - 1) * NBb + I) * BLK;
  };
  // row v's blocks go to slots DCH*(v&1) + j-1: each slot is used every
  // other row, so row v's phase parity is (v >> 1) & 1; a slot without a
  // block (v < j) completes its phase by a plain arrive
  auto slot_of = [&](int v, int j) { return DCH * (v & 1) + j - 1; };
  auto stage_row = [&](int v) {
    if (tid != 0 || v >= NBw) return;
    for (int j = 1; j <= DCH; ++j) {
      const int sl = slot_of(v, j);
      if (v >= j) stage_block(smem_u32(ring + sl * BLK), smem_u32(&sbar[sl]), blockp(v, j));
      else mbar_arrive(smem_u32(&sbar[sl]));
    }
  };
  // every thread waits for row v's slots (false: a copy did not land in time)
  auto wait_row = [&](int v) {
    bool ok = true;
    for (int j = 1; j <= DCH; ++j) ok = mbar_wait(smem_u32(&sbar[slot_of(v, j)]), (unsigned)((v >> 1) & 1)) && ok;
    return ok;
  };
  if (tid == 0) {
    bail = 0;
    for (int i = 0; i < RING; ++i) mbar_init(smem_u32(&sbar[i]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  stage_row(0);
  stage_row(1);
  auto wptr = [&](int v) { return wbuf + (long)(FWD ? v : NBw - 1 - v) * NB_ + c; };
  // w of the next row is polled one row ahead (a load that finds W_EMPTY
  // is repeated when the row comes)
  unsigned long long wnext = q == 0 ? ld_relaxed_u64(wptr(0)) : 0ull;
  for (int u = 0; u < NBw; ++u) {
    const int I = FWD ? u : NBw - 1 - u;
    const long gi = (long)I * NB_ + c;
    if (!wait_row(u) && atomicCAS(&bail, 0, 1) == 0) {
      err_note(err, TW_ERR_TIMEOUT, FWD ? 15 : 16);
      atomicExch(abort_flag, 1);
    }
    __syncthreads();
    if (bail) {                // row u+1 was staged too: let its copies land
      if (u + 1 < NBw) wait_row(u + 1);
      return;
    }
    // the product needs only z_{u-1} .. z_{u-DCH} and the staged blocks; a
    // w_u that was not there a row ago is polled again under the product
    unsigned long long wv = wnext;
    if (q == 0 && wv == W_EMPTY) wv = ld_relaxed_u64(wptr(u));
    if (q == 0 && u + 1 < NBw) wnext = ld_relaxed_u64(wptr(u + 1));
    {
      f2 S[DCH], T[DCH];
#pragma unroll
      for (int j = 1; j <= DCH; ++j) {
        S[j - 1] = f2_make(0.f, 0.f);
        T[j - 1] = S[j - 1];
        if (u < j) continue;
        const float *Ah = reinterpret_cast<const float *>(ring + slot_of(u, j) * BLK);
        const float *Al = Ah + BLK;
        const ZP *z = zp[(u - j) % DCH];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int k = kq * 8 + kk;
          const f2 ah = *reinterpret_cast<const f2 *>(Ah + k * NB_ + 2 * c2);
          const f2 al = *reinterpret_cast<const f2 *>(Al + k * NB_ + 2 * c2);
          const ZP zk = z[k];
          dacc_mac2(S[j - 1], T[j - 1], ah, al, zk.hh, zk.nn, zk.ll);
        }
      }
#pragma unroll
      for (int j = 2; j <= DCH; ++j) dd_add2(S[0], T[0], S[j - 1], T[j - 1]);
      const float2 sh = f2_split(S[0]), sl = f2_split(T[0]);
      red[kq][2 * c2] = dd_make_raw(sh.x, sl.x);
      red[kq][2 * c2 + 1] = dd_make_raw(sh.y, sl.y);
    }
    __syncthreads();           // partials in; row u's slots and z_{u-DCH} consumed
    stage_row(u + 2);          // into row u's slots
    if (q == 0) {
      const dd sum = dd_add(dd_add(dd_add(red[0][c], red[1][c]), dd_add(red[2][c], red[3][c])),
                            dd_add(dd_add(red[4][c], red[5][c]), dd_add(red[6][c], red[7][c])));
      if (wv == W_EMPTY) {
        const unsigned long long t0 = gtime();
        for (unsigned it = 1; (wv = ld_relaxed_u64(wbuf + gi)) == W_EMPTY; ++it) {
          if ((it & 63u) == 0 && (*(volatile int *)abort_flag || gtime() - t0 > WAIT_NS)) {
            if (!*(volatile int *)abort_flag) err_note(err, TW_ERR_TIMEOUT, FWD ? 11 : 12);
            atomicExch(abort_flag, 1);
            bail = 1;
            break;
          }
        }
      }
      dd z = dd_sub(bits_dd(wv), sum);
      if (gi >= nrows) z = dd_zero();
      out[gi] = dd_to_double(z);
      st_flag(outx + gi, z);   // the workers poll these entries
      ZP zz;                   // overwrites z_{u-DCH}
      zz.hh = f2_make(z.hi, z.hi);
      zz.nn = f2_make(-z.hi, -z.hi);
      zz.ll = f2_make(z.lo, z.lo);
      zz.pad = zz.ll;
      zp[u % DCH][c] = zz;
    }
    __syncthreads();
    if (bail) {                // rows u+1, u+2 were staged: let their copies land
      if (u + 1 < NBw) wait_row(u + 1);
      if (u + 2 < NBw) wait_row(u + 2);
      return;
    }
    // rows published so far: a hint for the workers' back-off, not a flag
    if (tid == 0) asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(progress), "r"(u + 1) : "memory");
  }
}

// ------------------------------------------------------------------ workers
// NZ entries of block row J of the solution (FWD at o + 16j, BWD at o + i),
// as stored: W_EMPTY where the chain has not reached them yet
template <bool FWD, int NZ>
__device__ __forceinline__ void zload(const dd *__restrict__ zx, int J, int o,
                                      unsigned long long (&zv)[NZ]) {
  const dd *p = zx + (long)J * NB_ + o;
#pragma unroll
  for (int i = 0; i < NZ; ++i) zv[i] = ld_relaxed_u64(p + (FWD ? 16 * i : i));
}
// poll the entries still W_EMPTY until they arrive; false after WAIT_NS or
// once the sweep is aborted
template <bool FWD, int NZ>
__device__ __forceinline__ bool zready(const dd *__restrict__ zx, int J, int o,
                                       unsigned long long (&zv)[NZ], const int *abort_flag) {
  const dd *p = zx + (long)J * NB_ + o;
  unsigned long long t0 = 0;
  for (unsigned it = 1;; ++it) {
    bool all = true;
#pragma unroll
    for (int i = 0; i < NZ; ++i) all = all && zv[i] != W_EMPTY;
    if (all) return true;
    // every missing entry again, the loads in flight together
#pragma unroll
    for (int i = 0; i < NZ; ++i)
      if (zv[i] == W_EMPTY) zv[i] = ld_relaxed_u64(p + (FWD ? 16 * i : i));
    if ((it & 63u) == 0) {
      if (*(volatile const int *)abort_flag) return false;
      const unsigned long long t = gtime();
      if (t0 == 0) t0 = t;
      else if (t - t0 > WAIT_NS) return false;
    }
  }
}

__device__ __forceinline__ double ld_b(const void *rhs, int kind, long i) {
  if (kind == 0) return __ldcg(reinterpret_cast<const double *>(rhs) + i);
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(rhs) + i);
  return (double)v.x + (double)v.y;
}

// A row's tasks other than its last (k < nk-1) store their partial vectors
// and count themselves done; the last task, which waits longest on the chain,
// adds the others' partials (in chunk order) while it waits and, after its
// own last dependency, stores w_u = that sum + its own partial directly.
template <bool FWD>
__device__ void worker_role(const dd *__restrict__ Lx, const double *__restrict__ Linv,
                            const void *__restrict__ rhs, int rhs_kind, const dd *__restrict__ zx,
                            const int2 *__restrict__ tasks, int ntasks, dd *__restrict__ part,
                            int maxk, int *cnt, dd *__restrict__ wbuf, int nrows, int NBw,
                            int *prog, int *err, int *abort_flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd *ring = reinterpret_cast<dd *>(smem_raw);          // [RING][64*64]
  __shared__ double sv[NB_];
  __shared__ dd spart[16][NB_ + 1];
  __shared__ dd sred[4][NB_];
  __shared__ dd spre[NB_];
  __shared__ double sinv[4][NB_];
  __shared__ __align__(8) unsigned long long sbar[RING];
  __shared__ int sT, sP, sbail, sready;
  const int tid = threadIdx.x;
  const int r_f = tid >> 2, q_f = tid & 3;        // FWD Linv product: row r, column quarter
  const int c_b = tid & 63, q_b = tid >> 6;       // BWD column c, row quarter
  const int g_f = tid >> 4, h_f = tid & 15;       // FWD rows 4g..4g+3, columns h + 16j
  const int r_p = tid & 63, q_p = tid >> 6;       // partial sums: row r, chunk class q
  int *progress = prog + 1;
  // blocks staged / consumed by this CTA so far: block number g sits in slot
  // g % RING and completes that slot's phase of parity (g / RING) & 1
  unsigned gstaged = 0, gused = 0;
  if (tid == 0) {
    for (int i = 0; i < RING; ++i) mbar_init(smem_u32(&sbar[i]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // let the staged but unconsumed copies land before the CTA leaves
  auto drain = [&]() {
    for (unsigned g = gused; g < gstaged; ++g) mbar_wait(smem_u32(&sbar[g % RING]), (g / RING) & 1);
  };
  for (;;) {
    __syncthreads();
    if (tid == 0) { sT = atomicAdd(prog, 1); sbail = 0; }
    __syncthreads();
    const int t = sT;
    if (t >= ntasks) return;
    const int u = tasks[t].x, k = tasks[t].y;
    const int I = FWD ? u : NBw - 1 - u;
    const int nk = row_tasks(u);
    const bool last = k == nk - 1;
    dd *pu = part + ((size_t)u * maxk) * NB_;
    // ---- this task's dependencies: d in [d0, d1)
    const int nd = u > DCH ? u - DCH : 0;
    const int d0 = k * CH, d1 = min(nd, d0 + CH);
    auto dblock = [&](int d) -> const dd * {
      const int J = FWD ? d : NBw - 1 - d;
      return Lx + (FWD ? packed_index(I, J) : packed_index(J, I)) * BLK;
    };
    auto stage = [&](int d) {    // uniform across the CTA; thread 0 issues
      const unsigned sl = gstaged % RING;
      if (tid == 0) stage_block(smem_u32(ring + sl * BLK), smem_u32(&sbar[sl]), dblock(d));
      ++gstaged;
    };
    // the other tasks' partials, added in chunk order: class q_p takes chunks
    // q_p, q_p+4, ... (eight loads in flight a thread), then the four class
    // sums are added in a fixed order
    auto presum = [&]() {
      dd s = dd_zero();
      for (int kb = q_p; kb < nk - 1; kb += 32) {
        dd v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int kk = kb + 4 * i;
          v[i] = kk < nk - 1 ? ld_dd_cg(pu + (size_t)kk * NB_ + r_p) : dd_zero();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) s = dd_add(s, v[i]);
      }
      sred[q_p][r_p] = s;
      __syncthreads();
      if (tid < NB_) spre[tid] = dd_add(dd_add(sred[0][tid], sred[1][tid]), dd_add(sred[2][tid], sred[3][tid]));
      __syncthreads();
    };
    // true once the other nk-1 tasks have stored their partials (thread 0)
    auto others_done = [&]() { return acq(cnt + u) >= nk - 1; };
    bool pre = !last || nk == 1;
    if (last && nk == 1 && tid < NB_) spre[tid] = dd_zero();
    // blocks d0 .. d0+RING-2 in flight
    for (int d = d0; d < min(d1, d0 + RING - 1); ++d) stage(d);
    dacc acc[4] = {dacc_zero(), dacc_zero(), dacc_zero(), dacc_zero()};
    int d = d0;
    while (d < d1) {
      // wait (with back-off) until the chain has published row d-1; the
      // entries of row d and later are then polled directly
      if (tid == 0) {
        int p = acq(progress);
        sready = 0;
        if (p < d && !pre && others_done()) {
          sready = 1;          // waiting anyway: add the others' partials first
        } else if (p < d) {
          const unsigned long long t0 = gtime();
          while ((p = acq(progress)) < d) {
            if (*(volatile int *)abort_flag) { sbail = 1; break; }
            if (gtime() - t0 > WAIT_NS) {
              err_note(err, TW_ERR_TIMEOUT, FWD ? 13 : 14);
              atomicExch(abort_flag, 1);
              sbail = 1;
              break;
            }
            if (!pre && others_done()) { sready = 1; break; }
            const int behind = d - p;
            __nanosleep(behind > 2 ? min(4096, 256 * (behind - 2)) : 32);
          }
        }
        sP = p;
      }
      __syncthreads();
      if (sbail) { drain(); return; }
      if (sready) { presum(); pre = true; continue; }
      const int dend = min(max(sP, d) + 1, d1);
      // this thread's z entries of dependency d (FWD 4 at h + 16j, BWD 16 at
      // 16q + i); the next dependency's are loaded while d's products run
      constexpr int NZ = FWD ? 4 : 16;
      const int zo = FWD ? h_f : q_b * 16;
      unsigned long long zc[NZ], zn[NZ];
      if (d < dend) zload<FWD, NZ>(zx, FWD ? d : NBw - 1 - d, zo, zc);
      for (; d < dend; ++d) {
        if (d + 1 < dend) zload<FWD, NZ>(zx, FWD ? d + 1 : NBw - 2 - d, zo, zn);
        if (!zready<FWD, NZ>(zx, FWD ? d : NBw - 1 - d, zo, zc, abort_flag) && atomicCAS(&sbail, 0, 1) == 0) {
          if (!*(volatile int *)abort_flag) err_note(err, TW_ERR_TIMEOUT, FWD ? 21 : 22);
          atomicExch(abort_flag, 1);
        }
        const unsigned sl = gused % RING;
        if (!mbar_wait(smem_u32(&sbar[sl]), (gused / RING) & 1) && atomicCAS(&sbail, 0, 1) == 0) {
          err_note(err, TW_ERR_TIMEOUT, FWD ? 17 : 18);
          atomicExch(abort_flag, 1);
        }
        __syncthreads();       // block d is in; every thread is done with block d-1's slot
        if (sbail) { drain(); return; }
        if (d + RING - 1 < d1) stage(d + RING - 1);   // into block d-1's slot
        const dd *A = ring + sl * BLK;
        ++gused;
        if (FWD) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) dacc_mac(acc[i], A[(g_f * 4 + i) * NB_ + h_f + 16 * j], bits_dd(zc[j]));
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) dacc_mac(acc[i & 1], A[(q_b * 16 + i) * NB_ + c_b], bits_dd(zc[i]));
        }
#pragma unroll
        for (int i = 0; i < NZ; ++i) zc[i] = zn[i];
      }
    }
    // ---- the last task: the others' partials, if the chain never kept it waiting
    if (!pre) {
      if (tid == 0) {
        const unsigned long long t0 = gtime();
        while (!others_done()) {
          if (*(volatile int *)abort_flag) { sbail = 1; break; }
          if (gtime() - t0 > WAIT_NS) {
            err_note(err, TW_ERR_TIMEOUT, FWD ? 19 : 20);
            atomicExch(abort_flag, 1);
            sbail = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      if (sbail) return;       // no copies in flight here
      presum();
    }
    // ---- chunk sum per row (64 values): row r = tid for tid < 64
    dd csum = dd_zero();
    if (FWD) {
#pragma unroll
      for (int i = 0; i < 4; ++i) spart[h_f][g_f * 4 + i] = dacc_get(acc[i]);
      __syncthreads();
      if (tid < NB_) {
        dd s = spart[0][tid];
#pragma unroll
        for (int h = 1; h < 16; ++h) s = dd_add(s, spart[h][tid]);
        csum = s;
      }
    } else {
      sred[q_b][c_b] = dd_add(dacc_get(acc[0]), dacc_get(acc[1]));
      __syncthreads();
      if (tid < NB_) csum = dd_add(dd_add(sred[0][tid], sred[1][tid]), dd_add(sred[2][tid], sred[3][tid]));
    }
    // ---- k = 0 also carries Linv_I b_I (FWD) / Linv_I^T y_I (BWD), in FP64
    dd res = dd_neg(csum);
    if (k == 0) {
      const long gb = (long)I * NB_ + tid;
      if (tid < NB_) sv[tid] = gb < nrows ? ld_b(rhs, rhs_kind, gb) : 0.0;
      __syncthreads();
      const double *iv = Linv + (size_t)I * BLK;
      double a2 = 0.0;
      if (FWD) {
        const double *p = iv + r_f * NB_ + q_f * 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) a2 = fma(__ldg(p + i), sv[q_f * 16 + i], a2);
        a2 += __shfl_xor_sync(0xffffffffu, a2, 1);
        a2 += __shfl_xor_sync(0xffffffffu, a2, 2);
        if (q_f == 0) sinv[0][r_f] = a2;
      } else {
        const double *p = iv + (q_b * 16) * NB_ + c_b;
#pragma unroll
        for (int i = 0; i < 16; ++i) a2 = fma(__ldg(p + i * NB_), sv[q_b * 16 + i], a2);
        sinv[q_b][c_b] = a2;
      }
      __syncthreads();
      if (tid < NB_) {
        const double b2 = FWD ? sinv[0][tid] : (sinv[0][tid] + sinv[1][tid]) + (sinv[2][tid] + sinv[3][tid]);
        res = dd_add(res, dd_from_double(b2));
      }
    }
    const long gw = (long)I * NB_ + tid;
    if (!last) {
      // ---- store the partial, then count the task done (release: the
      // barrier orders the stores before thread 0's fence and increment)
      if (tid < NB_) st_dd(pu + (size_t)k * NB_ + tid, res);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicAdd(cnt + u, 1);
      }
    } else if (tid < NB_) {
      // ---- w_u = the others' partials + this one: hand it to the chain
      st_flag(wbuf + gw, gw < nrows ? dd_add(spre[tid], res) : dd_zero());
    }
  }
}

template <bool FWD>
__global__ void __launch_bounds__(256, 1)   // one CTA per SM (192 KB ring)
k_trsv64(const dd *__restrict__ Lx, const double *__restrict__ Linv,
         const dd *__restrict__ bands, int NBb,
         const void *__restrict__ rhs, int rhs_kind, double *__restrict__ out, dd *__restrict__ outx,
         int nrows, int NBw, const int2 *__restrict__ tasks, int ntasks, dd *__restrict__ part,
         int maxk, int *cnt, dd *__restrict__ wbuf, int *prog, int *err, int *abort_flag) {
  if (blockIdx.x == 0)
    chain_role<FWD>(bands, NBb, wbuf, out, outx, nrows, NBw, prog + 1, err, abort_flag);
  else
    worker_role<FWD>(Lx, Linv, rhs, rhs_kind, outx, tasks, ntasks, part, maxk, cnt, wbuf, nrows,
                     NBw, prog, err, abort_flag);
}

// ------------------------------------------------------------- set-up kernels
// per packed block (I, J), J < I:  Lf = Linv_I L_IJ,  Lb = L_IJ Linv_J
__global__ void __launch_bounds__(256)
k_scale_blocks(const double *__restrict__ Lp, const double *__restrict__ Linv,
               dd *__restrict__ Lf, dd *__restrict__ Lb, int NB) {
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
    st_dd(Lf + (size_t)b * BLK + r * NB_ + c, dd_from_double(f));   // FP64 product, stored as float pairs
    st_dd(Lb + (size_t)b * BLK + r * NB_ + c, dd_from_double(g));
  }
}

// chain blocks as split planes (the 64x64 high parts, then the low parts),
// the layout of the packed products:
//   bands[0][j-1][I] = Lf_{I,I-j}^T (FWD, I >= j),  bands[1][j-1][I] = Lb_{I+j,I} (BWD, I+j < NB)
__global__ void k_bands(const dd *__restrict__ Lf, const dd *__restrict__ Lb, dd *__restrict__ bands,
                        int NB) {
  __shared__ dd t[NB_][NB_ + 1];
  const int I = blockIdx.x, j = blockIdx.y + 1;
  if (I >= j) {
    const dd *src = Lf + packed_index(I, I - j) * BLK;
    for (int i = threadIdx.x; i < BLK; i += blockDim.x) t[i / NB_][i % NB_] = src[i];
    __syncthreads();
    float *dst = reinterpret_cast<float *>(bands + ((size_t)(j - 1) * NB + I) * BLK);
    for (int i = threadIdx.x; i < BLK; i += blockDim.x) {
      const dd v = t[i % NB_][i / NB_];
      dst[i] = v.hi;
      dst[BLK + i] = v.lo;
    }
  }
  if (I + j < NB) {
    const dd *src = Lb + packed_index(I + j, I) * BLK;
    float *dst = reinterpret_cast<float *>(bands + ((size_t)(DCH + j - 1) * NB + I) * BLK);
    for (int i = threadIdx.x; i < BLK; i += blockDim.x) {
      const dd v = src[i];
      dst[i] = v.hi;
      dst[BLK + i] = v.lo;
    }
  }
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

int trsv64_chain_deps() { return DCH; }

cudaError_t launch_trsv64_setup(const double *Lp, const double *Linv, dd *Lf, dd *Lb, dd *bands,
                                int NB, cudaStream_t s) {
  if (NB <= 0) return cudaSuccess;
  const size_t sm = 3 * NB_ * (NB_ + 1) * sizeof(double);
  cudaFuncSetAttribute(k_scale_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const long nblk = (long)NB * (NB + 1) / 2;
  k_scale_blocks<<<(unsigned)nblk, 256, sm, s>>>(Lp, Linv, Lf, Lb, NB);
  count_launches(1);
  k_bands<<<dim3(NB, DCH), 256, 0, s>>>(Lf, Lb, bands, NB);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_trsv64(const Trsv64Args &a, bool fwd, cudaStream_t s) {
  if (a.NBw <= 0) return cudaSuccess;
  const size_t sm = RING * (size_t)BLK * sizeof(dd);
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
  if (e == cudaSuccess) e = cudaMemsetAsync(a.wbuf, 0xff, (size_t)a.NBw * NB_ * sizeof(dd), s);   // W_EMPTY
  if (e == cudaSuccess) e = cudaMemsetAsync(a.outx, 0xff, (size_t)a.NBw * NB_ * sizeof(dd), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.cnt, 0, a.NBw * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = std::min(a.ntasks + 1, res);
  if (fwd)
    k_trsv64<true><<<grid, 256, sm, s>>>(a.Lf, a.Linv, a.bands, a.NB, a.rhs, a.rhs_kind, a.out,
                                         a.outx, a.nrows, a.NBw, a.tasks, a.ntasks, a.part, a.maxk,
                                         a.cnt, a.wbuf, a.prog, a.err, a.abort_flag);
  else
    k_trsv64<false><<<grid, 256, sm, s>>>(a.Lb, a.Linv, a.bands + (size_t)DCH * a.NB * BLK, a.NB, a.rhs, a.rhs_kind, a.out,
                                          a.outx, a.nrows, a.NBw, a.tasks, a.ntasks, a.part, a.maxk,
                                          a.cnt, a.wbuf, a.prog, a.err, a.abort_flag);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tw
