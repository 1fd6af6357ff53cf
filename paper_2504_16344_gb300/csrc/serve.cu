// serve.cu -- the serving loop of Phase 4: replay a request trace against one
// context with continuous batching (policy in serve_policy.h).
//
// Each request names an event (its data vector sits in a device-resident
// bank) and a window Nt'.  A batch gathers its requests' data into slot
// buffers, runs the batched posterior mean + forecast (tw_infer_batch) and
// copies the forecasts to pinned host memory; the batch's completion time is
// its host enqueue time plus the device time between two events recorded
// around that work, and a request's latency is completion minus arrival.
// One batch is in flight at a time: the batched kernels fill the GPU.
#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "ctx.h"
#include "serve_policy.h"

using namespace tw;

namespace {

// d_slot[b] = bank[event[b]] for b < nb, rows of Nt*Nd doubles
__global__ void k_gather_rows(const double *__restrict__ bank, const int *__restrict__ ev,
                              double *__restrict__ dst, long row, int nb) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= row * nb) return;
  const int b = (int)(i / row);
  dst[i] = bank[(long)ev[b] * row + (i % row)];
}

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" {

tw_status tw_serve_simulate(int nreq, const double *arrival_s, int max_batch, double cost_ms,
                            double cost_ms_per_req, double *latency_ms, int *batch_of) {
  if (nreq < 0 || max_batch < 1 || (nreq > 0 && (!arrival_s || !latency_ms))) return TW_ERR_ARG;
  for (int i = 1; i < nreq; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) return TW_ERR_ARG;
  twserve::Policy pol(nreq, arrival_s, max_batch);
  double t = nreq ? arrival_s[0] : 0.0;
  int nb_id = 0;
  while (!pol.done()) {
    pol.admit(t);
    if (!pol.waiting()) { t = pol.next_arrival(); continue; }
    int first, count;
    pol.take(&first, &count);
    const double t_end = t + 1e-3 * (cost_ms + cost_ms_per_req * count);
    for (int i = first; i < first + count; ++i) {
      latency_ms[i] = 1e3 * (t_end - arrival_s[i]);
      if (batch_of) batch_of[i] = nb_id;
    }
    ++nb_id;
    t = t_end;
  }
  return TW_OK;
}

tw_status tw_serve_replay(tw_ctx *c, tw_prec prec, int nreq, const double *arrival_s,
                          const int *event, const int *window, int nevents,
                          const double *event_data, int max_batch, double *latency_ms,
                          double *q_out, double *m_out, tw_serve_stats *stats, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nreq < 0 || nevents < 1 || !event_data ||
      (nreq > 0 && (!arrival_s || !event || !window || !latency_ms)))
    return twh::fail(c, TW_ERR_ARG, "bad trace arguments");
  if (max_batch < 1 || max_batch > c->bmax)
    return twh::fail(c, TW_ERR_ARG, "max_batch must be in [1, reserved batch]");
  if (!stream) return twh::fail(c, TW_ERR_ARG, "serving needs a created stream");
  for (int i = 0; i < nreq; ++i) {
    if (event[i] < 0 || event[i] >= nevents) return twh::fail(c, TW_ERR_ARG, "event out of range");
    if (window[i] < 1 || window[i] > c->Nt) return twh::fail(c, TW_ERR_ARG, "window must be in [1, Nt]");
    if (i > 0 && arrival_s[i] < arrival_s[i - 1])
      return twh::fail(c, TW_ERR_ARG, "arrivals must be sorted");
  }
  cudaStream_t s = (cudaStream_t)stream;
  TW_CUDA(c, cudaSetDevice(c->dev));
  const int Nt = c->Nt, Nd = c->Nd, Nm = c->Nm, Nq = c->Nq;
  const size_t B = max_batch;
  const long drow = (long)Nt * Nd;
  // session buffers (set-up, before the clock starts)
  double *d_slot = (double *)twh::dalloc(c, B * drow * sizeof(double));
  double *m_slot = (double *)twh::dalloc(c, B * (size_t)Nt * Nm * sizeof(double));
  double *q_slot = (double *)twh::dalloc(c, B * (size_t)Nt * Nq * sizeof(double));
  int *idx_dev = (int *)twh::dalloc(c, 2 * B * sizeof(int));
  int *idx_host = nullptr;
  double *q_host = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  auto cleanup = [&]() {
    twh::dfree(c, d_slot); twh::dfree(c, m_slot); twh::dfree(c, q_slot); twh::dfree(c, idx_dev);
    if (idx_host) cudaFreeHost(idx_host);
    if (q_host) cudaFreeHost(q_host);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  };
  if (!d_slot || !m_slot || !q_slot || !idx_dev) { cleanup(); return twh::fail(c, TW_ERR_OOM, "serving slots"); }
  if (cudaMallocHost(&idx_host, 2 * B * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&q_host, B * (size_t)Nt * Nq * sizeof(double)) != cudaSuccess ||
      cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) {
    cleanup();
    return twh::fail(c, TW_ERR_OOM, "pinned staging / events");
  }
  twserve::Policy pol(nreq, arrival_s, max_batch);
  int batches = 0, maxb = 0;
  double busy = 0.0, t_last = 0.0;
  tw_status st = TW_OK;
  const auto t0 = std::chrono::steady_clock::now();
  while (!pol.done()) {
    pol.admit(now_s(t0));
    if (!pol.waiting()) {
      // idle: sleep until the next arrival (short naps keep the clock honest)
      const double wait = pol.next_arrival() - now_s(t0);
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 2e-4)));
      continue;
    }
    int first, count;
    pol.take(&first, &count);
    for (int k = 0; k < count; ++k) {
      idx_host[k] = event[first + k];
      idx_host[B + k] = window[first + k];
    }
    const double t_enq = now_s(t0);
    if (cudaEventRecord(ev0, s) != cudaSuccess ||
        cudaMemcpyAsync(idx_dev, idx_host, 2 * B * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      st = twh::fail(c, TW_ERR_CUDA, "serving: enqueue");
      break;
    }
    const long tot = drow * count;
    k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(event_data, idx_dev, d_slot, drow, count);
    count_launches(1);
    st = tw_infer_batch(c, prec, count, idx_dev + B, d_slot, m_slot, q_slot, stream);
    if (st != TW_OK) break;
    if (cudaMemcpyAsync(q_host, q_slot, (size_t)count * Nt * Nq * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaEventRecord(ev1, s) != cudaSuccess) {
      st = twh::fail(c, TW_ERR_CUDA, "serving: result copy");
      break;
    }
    // wait for the batch while admitting arrivals
    while (cudaEventQuery(ev1) == cudaErrorNotReady) {
      pol.admit(now_s(t0));
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) {
      st = twh::fail(c, TW_ERR_CUDA, "serving: batch timing");
      break;
    }
    const double t_done = t_enq + 1e-3 * ms;
    busy += 1e-3 * ms;
    t_last = std::max(t_last, t_done);
    for (int k = 0; k < count; ++k) latency_ms[first + k] = 1e3 * (t_done - arrival_s[first + k]);
    if (q_out)
      std::copy(q_host, q_host + (size_t)count * Nt * Nq, q_out + (size_t)first * Nt * Nq);
    if (m_out &&
        cudaMemcpy(m_out + (size_t)first * Nt * Nm, m_slot, (size_t)count * Nt * Nm * sizeof(double),
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = twh::fail(c, TW_ERR_CUDA, "serving: m copy");
      break;
    }
    ++batches;
    maxb = std::max(maxb, count);
  }
  if (st == TW_OK) st = tw_check(c, stream);
  if (stats) {
    stats->batches = batches;
    stats->max_batch = maxb;
    stats->mean_batch = batches ? (double)nreq / batches : 0.0;
    stats->makespan_s = nreq ? t_last - arrival_s[0] : 0.0;
    stats->busy_s = busy;
  }
  cleanup();
  return st;
}

}  // extern "C"
