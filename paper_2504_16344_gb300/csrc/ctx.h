// ctx.h -- the tw_ctx structure and host helpers shared by the API files.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/tw.h"
#include "kernels.h"

// One set of batch workspaces ("lane"), RHS-major: a batch of up to bmax
// right-hand sides runs in it.  The context's reserved batch is one lane;
// the serving loop adds lanes so that several batches run at the same time.
struct tw_lane {
  int bmax = 0;
  int *win_dev = nullptr;            // [bmax] windows of host-window batched calls
  int *trsm_prog = nullptr;          // [2][trsm_prog_ints(bmax)] solve counters
  double *bz = nullptr, *by = nullptr;      // [bmax][n_pad] FP64 solves
  tw::dd *bzd = nullptr, *byd = nullptr;    // [bmax][n_pad] float-pair solves (mixed)
  double *brd = nullptr;             // [bmax][Nt][Nd] data-side scratch (samples)
  void *byh = nullptr;               // [bmax][Nf][Rmax] data-side spectra (16-byte entries)
  void *bxh = nullptr;               // [bmax][Nf][Nm] parameter-side spectra / prior work
  void *bpart = nullptr;             // [bmax][Nf][nchunk][Rmax] forward-product partial sums
  // data-side slices and column exponents of the tensor-core adjoint (sized
  // for any tile of up to 80 right-hand sides)
  void *bsl_ws = nullptr;
  int *bsl_eb = nullptr;
  size_t bsl_ws_n = 0, bsl_eb_n = 0;
  // tiles of the batched products (tw_batch_tiles): right-hand sides per
  // tensor-core tile (mixed adjoint) and per warp (FP64-class adjoint), lanes
  // per right-hand side (forward products); chosen by measurement at
  // tw_reserve_batch, the same for every lane of a context
  int sl_tile = 0;
  int adj_rw = 0;
  int fwd_lpb = 1;
  size_t bytes = 0;                  // device bytes of the lane
};

struct tw_ctx {
  int dev = 0;
  int Nd = 0, Nq = 0, Nx = 0, Ny = 0, Nt = 0, Nm = 0, Nf = 0, Rmax = 0;
  double Lx = 1.0, Ly = 1.0;
  unsigned keep = 0;
  // frequency-domain operators op[which][fmt], [Nf][rows][Nm]
  void *op[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  // G^ = F^ C per frequency (the paper's G* = Gamma_pr F* of Phase 2), per kept
  // format, when TW_KEEP_G: the adjoint applies of tw_infer then need no prior filter
  void *opG[3] = {nullptr, nullptr, nullptr};
  // row exponents of the FP32 storages for the batched adjoint on the tensor
  // cores: ea[which][fmt][w][m] (fmt 1, 2), eaG[fmt] for G^ (gemm_sl.cu)
  int8_t *ea[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int8_t *eaG[3] = {nullptr, nullptr, nullptr};
  std::vector<char> loaded[2];     // per row: loaded?
  std::vector<unsigned long long> col_hash;   // per row of F: fingerprint of its block column
  // FFT plans and twiddle tables (df64 and float)
  tw::FftPlan plT{}, plX{}, plY{};
  tw::cdd *twT = nullptr, *twL = nullptr, *twX = nullptr, *twY = nullptr;
  tw::cf *twTf = nullptr, *twLf = nullptr, *twXf = nullptr, *twYf = nullptr;
  tw::cd *twXd = nullptr, *twYd = nullptr;      // native FP64 tables (set-up filters)
  // prior: lambda^power / N, power 1 and 1/2
  bool prior_set = false;
  double nu = 1, ell = 0.1, var = 1;
  tw::dd *lam1 = nullptr, *lamh = nullptr;
  float *lam1f = nullptr, *lamhf = nullptr;
  double *lamhd = nullptr;                        // sqrt(lambda) / N in FP64
  double *lam1d = nullptr;                        // lambda / N in FP64 (forming G^)
  // G = Phi C^{1/2} (rows t*Nd + sensor), built in FP64 from the loaded
  // block column when the prior is already set; consumed by tw_factor_K
  tw::dd *G = nullptr;
  std::vector<char> g_rows;
  // online workspaces
  tw::cdd *wf = nullptr;    // [Nf][Nm]
  tw::cdd *wr = nullptr;    // [Nf][Rmax]
  tw::cdd *part = nullptr;  // [Nf][nchunk][Rmax]
  tw::dd *wt = nullptr;     // [Nt][Nm]
  tw::cdd *ws = nullptr;    // [ceil(Nt/2)][Nm]
  int *d_err = nullptr;     // device error record: [0] code, [1] info
  // data-space Hessian K = sigma^2 I + F Gamma_pr F^T and its factors
  int n = 0, n_pad = 0, NB = 0;
  double sigma2 = 0.0, shift32 = 0.0;
  bool have64 = false, have32 = false;
  double *Lp64 = nullptr, *inv64 = nullptr;                      // FP64 factor, packed 64x64 blocks
  double *chF64 = nullptr, *chB64 = nullptr;                      // chain blocks of the solves
  // single-vector FP64-class solves (trsv64.cu): block-scaled factor as
  // float pairs and scheduling state
  tw::dd *Lfs = nullptr, *Lbs = nullptr;                          // packed, like Lp64
  tw::dd *bands = nullptr;                                        // [2][DCH][NB][64][64] chain blocks
  int2 *tasks = nullptr;                                          // worker task table
  std::vector<int> task_prefix;                                   // tasks of rows < u: task_prefix[u]
  tw::dd *tpart = nullptr;                                        // [NB][maxk][64]
  int tmaxk = 0;
  int *tcnt = nullptr;                                            // [NB]
  tw::dd *wbufx = nullptr;                                        // [n_pad]
  tw::dd *zx = nullptr;                                           // [n_pad] sweep output, float pairs
  tw::dd *Kp64 = nullptr;                                         // K, packed, double-float
  float *Lp32 = nullptr, *inv32 = nullptr;
  float *chF32 = nullptr, *chB32 = nullptr;
  // solve workspaces
  tw::dd *vz = nullptr, *vy = nullptr, *vr = nullptr;          // [n_pad]
  double *zd = nullptr, *yd = nullptr, *rd = nullptr, *ad = nullptr;   // [n_pad]
  float *fz = nullptr, *fy = nullptr;                          // [n_pad]
  int *counter = nullptr;     // [4]: forward (ticket, rows done), backward (ticket, rows done)
  int *abort_flag = nullptr;
  double *d_norm = nullptr;
  int ir_steps = 3;
  int solver = TW_SOLVE_FACTOR64;
  double ir_probe_resid = 0.0;
  // batched right-hand sides (tw_reserve_batch): the reserved lane and the
  // tiles chosen for its products
  tw_lane lane;
  tw_tiles tiles{};
  tw::dd *inv_dd = nullptr;   // float-pair diagonal-block inverses of the FP64 factor (batched solves)
  // Phase 3 QoI precomputations (tw_qoi_build): rows indexed by QoI entry t*Nq + i
  double *Qmap = nullptr, *Wmap = nullptr;   // [Nq Nt][Nd Nt]: Q = F_q Gamma_pr F^T K^-1, W = (F Gamma_pr F_q^T)^T
  double *Cqq = nullptr;                     // [Nq Nt][Nq Nt]: F_q Gamma_pr F_q^T
  double *qvar = nullptr;                    // [Nq Nt]: diagonal of the QoI posterior covariance
  bool have_qoi = false;
  // per-phase timing
  struct PhaseEv { int ph; cudaEvent_t a, b; };
  bool prof = false;
  std::vector<PhaseEv> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[TW_PH_COUNT] = {0};
  long long prof_calls[TW_PH_COUNT] = {0};
  size_t bytes = 0;
  std::string err;
  std::vector<void *> allocs;
  std::vector<size_t> alloc_sizes;
};

namespace twh {

// Times one phase with two events on `s` when profiling is on (RAII).
struct Phase {
  tw_ctx *c;
  int ph;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Phase(tw_ctx *c_, int ph_, cudaStream_t s_);
  ~Phase();
};

tw_status fail(tw_ctx *c, tw_status st, const std::string &msg);
tw_status cuda_fail(tw_ctx *c, cudaError_t e, const char *where);
void *dalloc(tw_ctx *c, size_t bytes);   // tracked cudaMalloc; nullptr on failure
void dfree(tw_ctx *c, void *p);
tw::FftPlan make_plan(int M);
// fingerprint of F's whole block column (from the per-row ones)
unsigned long long column_fingerprint(const tw_ctx *c);
// batch copies after a factorisation: the float-pair factor for mixed batched
// solves and the tensor-core operator tiles (no-op unless reserved)
tw_status refresh_dd_factor(tw_ctx *c, cudaStream_t s);

}  // namespace twh

// host-window calls routed to the batched path (tw_batch.cu)
namespace twb {
// allocate / free a lane's workspaces (bmax right-hand sides)
tw_status alloc_lane(tw_ctx *c, tw_lane &L, int bmax);
void free_lane(tw_ctx *c, tw_lane &L);
size_t lane_bytes(const tw_ctx *c, int bmax);
// the batched posterior mean (+ forecast when q) of B right-hand sides in lane L
tw_status infer_core(tw_ctx *c, tw_lane &L, tw_prec prec, int B, const int *win, const double *rhs,
                     long rhs_bstride, double *m, double *q, cudaStream_t s);
// measure the tile candidates of the batched products on lane L (or take
// them from the process-wide cache of earlier contexts with the same shapes)
tw_status autotune_lane(tw_ctx *c, tw_lane &L);
void copy_tiles(tw_lane &dst, const tw_lane &src);
tw_status infer_host_windows(tw_ctx *c, tw_prec prec, int nrhs, const int *nt_window,
                             const double *d, double *m, cudaStream_t s);
tw_status sample_host_windows(tw_ctx *c, int ns, const int *nt_window, const double *d,
                              const double *z_m, const double *z_n, double sigma, double *samples,
                              cudaStream_t s);
tw_status forecast_full(tw_ctx *c, tw_prec prec, int nrhs, const double *m, double *q,
                        cudaStream_t s);
}  // namespace twb

#define TW_CUDA(c, call)                                             \
  do {                                                               \
    cudaError_t _e = (call);                                         \
    if (_e != cudaSuccess) return twh::cuda_fail((c), _e, #call);    \
  } while (0)
