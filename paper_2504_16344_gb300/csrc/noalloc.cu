// noalloc.cu -- tw_p2o_apply_noalloc: the forward Toeplitz apply with the
// per-chunk partial sums of the frequency GEMV kept in a fixed device array.
//
// Callers that run where device memory may not be allocated (a real-time loop
// with a fixed memory footprint, a host that forbids allocation after start-up,
// code that must not enter the CUDA allocator) can use this entry point: the
// call itself allocates nothing.  It reuses the library's kernels and the
// context's FFT buffers (allocated once by tw_create); only the GEMV's
// partial-sum scratch, which tw_p2o_apply takes from the context, comes from
// the file-scope array below instead.
#include <stdio.h>

#include <mutex>

#include "ctx.h"

using namespace tw;

namespace {

// Fixed scratch for the GEMV partial sums: [Nt+1][ceil(Nm/1024)][rows] complex
// entries of 16 bytes (FP64 path) or 8 bytes (FP32 paths).  Every GPU that
// loads the library holds these 32 MiB until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// once per device with that device current.
constexpr int kMaxDevices = 64;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

tw_status scratch_for_device(tw_ctx *c, void **out) {
  if (c->dev < 0 || c->dev >= kMaxDevices) return twh::fail(c, TW_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[c->dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return twh::cuda_fail(c, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[c->dev] = p;
  }
  *out = g_scratch_ptr[c->dev];
  return TW_OK;
}

}  // namespace

extern "C" tw_status tw_p2o_apply_noalloc(tw_ctx *c, tw_map which, tw_prec prec, int nrhs,
                                          const double *x, double *out, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (which != TW_MAP_F && which != TW_MAP_FQ) return twh::fail(c, TW_ERR_ARG, "bad map");
  if (prec < 0 || prec > 2 || !c->op[which][prec])
    return twh::fail(c, TW_ERR_ARG, "requested precision was not kept at tw_create");
  for (char l : c->loaded[which])
    if (!l) return twh::fail(c, TW_ERR_STATE, "block column not fully loaded");
  if (nrhs < 0 || (nrhs > 0 && (!x || !out))) return twh::fail(c, TW_ERR_ARG, "bad rhs");
  const int R = which == TW_MAP_F ? c->Nd : c->Nq;
  const int Nt = c->Nt, Nf = c->Nf, Nm = c->Nm;
  const size_t elem = prec == TW_PREC_FP64 ? sizeof(cdd) : sizeof(cf);
  const size_t need = (size_t)Nf * gemv_fwd_nchunk(Nm) * R * elem;
  if (need > kNoAllocScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "tw_p2o_apply_noalloc: the GEMV partial sums need %zu bytes, above the fixed %zu-byte "
             "scratch; use tw_p2o_apply", need, kNoAllocScratchBytes);
    return twh::fail(c, TW_ERR_ARG, buf);
  }
  TW_CUDA(c, cudaSetDevice(c->dev));
  void *scratch = nullptr;
  tw_status st = scratch_for_device(c, &scratch);
  if (st != TW_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const void *A = c->op[which][prec];
  // every partial sum is written before it is read, so the array needs no clearing
  for (int r = 0; r < nrhs; ++r) {
    const double *xr = x + (size_t)r * Nt * Nm;
    double *outr = out + (size_t)r * Nt * R;
    if (prec == TW_PREC_FP64) {
      TW_CUDA(c, launch_rfft_time_dd(xr, 0, Nm, Nt, c->wf, Nm, Nm, c->plT, c->twT, c->twL, s));
      TW_CUDA(c, launch_gemv_fwd_dd(A, FMT_DD, c->wf, (cdd *)scratch, c->wr, Nf, R, Nm, s));
      TW_CUDA(c, launch_irfft_time_dd(c->wr, R, outr, 0, R, R, Nt, c->plT, c->twT, c->twL, s));
    } else {
      cf *wf = (cf *)c->wf, *wr = (cf *)c->wr;
      TW_CUDA(c, launch_rfft_time_f(xr, 0, Nm, Nt, wf, Nm, Nm, c->plT, c->twTf, c->twLf, s));
      TW_CUDA(c, launch_gemv_fwd_f(A, (int)prec, wf, (cf *)scratch, wr, Nf, R, Nm, s));
      TW_CUDA(c, launch_irfft_time_f(wr, R, outr, 0, R, R, Nt, c->plT, c->twTf, c->twLf, s));
    }
  }
  return TW_OK;
}
