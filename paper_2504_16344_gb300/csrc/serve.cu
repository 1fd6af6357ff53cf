// serve.cu -- the serving loop of Phase 4: replay a request trace against one
// context with continuous batching (policy in serve_policy.h).
//
// Each request names an event (its data vector sits in a device-resident
// bank) and a window Nt'.  A batch gathers its requests' data into its
// lane's slot buffers, runs the batched posterior mean + forecast in that
// lane's workspaces on the lane's own stream and copies the forecasts to
// pinned host memory.  Several lanes are in flight at once: a request that
// arrives while batches run starts as soon as any lane is free, and its
// kernels overlap the running batches' on the device.  Lane 0 is the
// context's reserved batch; the session adds lanes while device memory
// allows (up to the requested count).  Completion times come from device
// events against one reference event recorded when the clock starts; a
// request's latency is its batch's completion minus its arrival.
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

// one lane of a serving session: workspaces, slot buffers, stream, staging
struct ServeLane {
  tw_lane *work = nullptr;        // the batch workspaces (lane 0: the context's)
  bool owned = false;             // workspaces allocated by the session
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double *d_slot = nullptr, *m_slot = nullptr, *q_slot = nullptr;
  int *idx_dev = nullptr, *idx_host = nullptr;
  double *q_host = nullptr;
  cudaEvent_t done = nullptr;
  int first = 0, count = 0;       // the batch in flight
};

constexpr int MAX_LANES = 4;

}  // namespace

extern "C" {

tw_status tw_serve_simulate(int nreq, const double *arrival_s, int max_batch, int lanes,
                            double cost_ms, double cost_ms_per_req, double *latency_ms,
                            int *batch_of) {
  if (nreq < 0 || max_batch < 1 || lanes < 1 || (nreq > 0 && (!arrival_s || !latency_ms)))
    return TW_ERR_ARG;
  for (int i = 1; i < nreq; ++i)
    if (arrival_s[i] < arrival_s[i - 1]) return TW_ERR_ARG;
  twserve::Policy pol(nreq, arrival_s, max_batch, lanes);
  std::vector<double> end(lanes, 0.0);
  std::vector<int> first(lanes, 0), count(lanes, 0);
  double t = nreq ? arrival_s[0] : 0.0;
  int nb_id = 0;
  while (!pol.done()) {
    pol.admit(t);
    // every free lane takes a batch while requests wait
    int l;
    while (pol.waiting() && (l = pol.free_lane()) >= 0) {
      pol.take(l, &first[l], &count[l]);
      end[l] = t + 1e-3 * (cost_ms + cost_ms_per_req * count[l]);
      for (int i = first[l]; i < first[l] + count[l]; ++i)
        if (batch_of) batch_of[i] = nb_id;
      ++nb_id;
    }
    // advance to the next event: a batch finishing or a request arriving
    const double inf = 1e300;
    const double t_arr = pol.all_taken() || pol.next_arrival() < 0 ? inf : pol.next_arrival();
    int l_end = -1;
    for (int k = 0; k < lanes; ++k)
      if (count[k] > 0 && (l_end < 0 || end[k] < end[l_end])) l_end = k;
    const double t_end = l_end < 0 ? inf : end[l_end];
    if (t_end <= t_arr) {
      t = t_end;
      for (int i = first[l_end]; i < first[l_end] + count[l_end]; ++i)
        latency_ms[i] = 1e3 * (t - arrival_s[i]);
      count[l_end] = 0;
      pol.release(l_end);
    } else if (t_arr < inf) {
      t = std::max(t, t_arr);
    }
  }
  return TW_OK;
}

tw_status tw_serve_replay(tw_ctx *c, tw_prec prec, int nreq, const double *arrival_s,
                          const int *event, const int *window, int nevents,
                          const double *event_data, int max_batch, int lanes, double *latency_ms,
                          double *q_out, double *m_out, tw_serve_stats *stats, void *stream) {
  if (!c) return TW_ERR_ARG;
  if (nreq < 0 || nevents < 1 || !event_data ||
      (nreq > 0 && (!arrival_s || !event || !window || !latency_ms)))
    return twh::fail(c, TW_ERR_ARG, "bad trace arguments");
  if (max_batch < 1 || max_batch > c->lane.bmax)
    return twh::fail(c, TW_ERR_ARG, "max_batch must be in [1, reserved batch]");
  if (lanes < 0 || lanes > MAX_LANES) return twh::fail(c, TW_ERR_ARG, "lanes must be in [0, 4]");
  if (!stream) return twh::fail(c, TW_ERR_ARG, "serving needs a created stream");
  for (int i = 0; i < nreq; ++i) {
    if (event[i] < 0 || event[i] >= nevents) return twh::fail(c, TW_ERR_ARG, "event out of range");
    if (window[i] < 1 || window[i] > c->Nt) return twh::fail(c, TW_ERR_ARG, "window must be in [1, Nt]");
    if (i > 0 && arrival_s[i] < arrival_s[i - 1])
      return twh::fail(c, TW_ERR_ARG, "arrivals must be sorted");
  }
  TW_CUDA(c, cudaSetDevice(c->dev));
  TW_CUDA(c, cudaDeviceSynchronize());
  const int Nt = c->Nt, Nd = c->Nd, Nm = c->Nm, Nq = c->Nq;
  const size_t B = max_batch;
  const long drow = (long)Nt * Nd;
  const size_t slot_bytes = B * ((size_t)drow + (size_t)Nt * Nm + (size_t)Nt * Nq) * sizeof(double) +
                            2 * B * sizeof(int);
  // lanes: the reserved batch, plus more while device memory allows (up to
  // `lanes`, 0 = as many as fit, at most four), with a 2 GB margin
  const int want = lanes == 0 ? MAX_LANES : lanes;
  std::vector<ServeLane> L(1);
  L[0].work = &c->lane;
  L[0].stream = (cudaStream_t)stream;
  tw_status st = TW_OK;
  cudaEvent_t ev_ref = nullptr;
  auto cleanup = [&]() {
    for (ServeLane &l : L) {
      twh::dfree(c, l.d_slot); twh::dfree(c, l.m_slot); twh::dfree(c, l.q_slot); twh::dfree(c, l.idx_dev);
      if (l.idx_host) cudaFreeHost(l.idx_host);
      if (l.q_host) cudaFreeHost(l.q_host);
      if (l.done) cudaEventDestroy(l.done);
      if (l.own_stream) cudaStreamDestroy(l.stream);
      if (l.owned) { twb::free_lane(c, *l.work); delete l.work; }
    }
    if (ev_ref) cudaEventDestroy(ev_ref);
  };
  // extra lanes copy the reserved lane's size: the batched kernels' tiling
  // follows it, and a result must not depend on the lane it ran in
  const size_t lane_need = twb::lane_bytes(c, c->lane.bmax) + slot_bytes;
  while ((int)L.size() < want) {
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) break;
    // this lane's slots and the next lane's workspaces must fit beside a margin
    if (freeb < slot_bytes * L.size() + lane_need + ((size_t)2 << 30)) break;
    ServeLane l;
    l.work = new tw_lane();
    l.owned = true;
    if (twb::alloc_lane(c, *l.work, c->lane.bmax) != TW_OK) {
      delete l.work;
      break;
    }
    twb::copy_tiles(*l.work, c->lane);
    if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess) {
      twb::free_lane(c, *l.work);
      delete l.work;
      break;
    }
    l.own_stream = true;
    L.push_back(l);
  }
  cudaGetLastError();
  for (ServeLane &l : L) {
    l.d_slot = (double *)twh::dalloc(c, B * drow * sizeof(double));
    l.m_slot = (double *)twh::dalloc(c, B * (size_t)Nt * Nm * sizeof(double));
    l.q_slot = (double *)twh::dalloc(c, B * (size_t)Nt * Nq * sizeof(double));
    l.idx_dev = (int *)twh::dalloc(c, 2 * B * sizeof(int));
    if (!l.d_slot || !l.m_slot || !l.q_slot || !l.idx_dev ||
        cudaMallocHost(&l.idx_host, 2 * B * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&l.q_host, B * (size_t)Nt * Nq * sizeof(double)) != cudaSuccess ||
        cudaEventCreate(&l.done) != cudaSuccess) {
      cleanup();
      return twh::fail(c, TW_ERR_OOM, "serving slots / pinned staging / events");
    }
  }
  if (cudaEventCreate(&ev_ref) != cudaSuccess) {
    cleanup();
    return twh::fail(c, TW_ERR_CUDA, "serving: reference event");
  }
  const int nl = (int)L.size();
  twserve::Policy pol(nreq, arrival_s, max_batch, nl);
  int batches = 0, maxb = 0, max_inflight = 0;
  double busy = 0.0, t_last = 0.0;
  std::vector<double> t_start(nl, 0.0);
  TW_CUDA(c, cudaDeviceSynchronize());
  const auto t0 = std::chrono::steady_clock::now();
  if (cudaEventRecord(ev_ref, L[0].stream) != cudaSuccess || cudaEventSynchronize(ev_ref) != cudaSuccess) {
    cleanup();
    return twh::fail(c, TW_ERR_CUDA, "serving: reference event");
  }
  const double t_ref = now_s(t0);     // host time of the device reference point
  while (!pol.done() && st == TW_OK) {
    bool progressed = false;
    // completions
    for (int k = 0; k < nl && st == TW_OK; ++k) {
      ServeLane &l = L[k];
      if (l.count == 0 || cudaEventQuery(l.done) != cudaSuccess) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev_ref, l.done) != cudaSuccess) {
        st = twh::fail(c, TW_ERR_CUDA, "serving: batch timing");
        break;
      }
      const double t_done = t_ref + 1e-3 * ms;
      busy += std::max(0.0, t_done - t_start[k]);
      t_last = std::max(t_last, t_done);
      for (int i = 0; i < l.count; ++i) latency_ms[l.first + i] = 1e3 * (t_done - arrival_s[l.first + i]);
      if (q_out)
        std::copy(l.q_host, l.q_host + (size_t)l.count * Nt * Nq, q_out + (size_t)l.first * Nt * Nq);
      if (m_out && cudaMemcpy(m_out + (size_t)l.first * Nt * Nm, l.m_slot,
                              (size_t)l.count * Nt * Nm * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = twh::fail(c, TW_ERR_CUDA, "serving: m copy");
        break;
      }
      l.count = 0;
      pol.release(k);
      progressed = true;
    }
    if (st != TW_OK) break;
    // launches: every free lane takes the oldest waiting requests
    pol.admit(now_s(t0));
    int k;
    while (st == TW_OK && pol.waiting() && (k = pol.free_lane()) >= 0) {
      ServeLane &l = L[k];
      pol.take(k, &l.first, &l.count);
      for (int i = 0; i < l.count; ++i) {
        l.idx_host[i] = event[l.first + i];
        l.idx_host[B + i] = window[l.first + i];
      }
      t_start[k] = std::max(now_s(t0), t_ref);
      if (cudaMemcpyAsync(l.idx_dev, l.idx_host, 2 * B * sizeof(int), cudaMemcpyHostToDevice, l.stream) !=
          cudaSuccess) {
        st = twh::fail(c, TW_ERR_CUDA, "serving: enqueue");
        break;
      }
      const long tot = drow * l.count;
      k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, l.stream>>>(event_data, l.idx_dev, l.d_slot,
                                                                          drow, l.count);
      count_launches(1);
      st = twb::infer_core(c, *l.work, prec, l.count, l.idx_dev + B, l.d_slot, drow, l.m_slot, l.q_slot,
                           l.stream);
      if (st != TW_OK) break;
      if (cudaMemcpyAsync(l.q_host, l.q_slot, (size_t)l.count * Nt * Nq * sizeof(double),
                          cudaMemcpyDeviceToHost, l.stream) != cudaSuccess ||
          cudaEventRecord(l.done, l.stream) != cudaSuccess) {
        st = twh::fail(c, TW_ERR_CUDA, "serving: result copy");
        break;
      }
      ++batches;
      maxb = std::max(maxb, l.count);
      max_inflight = std::max(max_inflight, pol.in_flight());
      progressed = true;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (st != TW_OK) {
    for (ServeLane &l : L) cudaStreamSynchronize(l.stream);
  }
  for (ServeLane &l : L)
    if (st == TW_OK) st = tw_check(c, l.stream);
  if (stats) {
    stats->batches = batches;
    stats->max_batch = maxb;
    stats->mean_batch = batches ? (double)nreq / batches : 0.0;
    stats->makespan_s = nreq ? t_last - arrival_s[0] : 0.0;
    stats->busy_s = busy;
    stats->lanes = nl;
    stats->max_in_flight = max_inflight;
  }
  cleanup();
  return st;
}

}  // extern "C"
