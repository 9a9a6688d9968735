// Launch accounting of the wfft kernels: every launch is counted per kernel
// kind and precision; when profiling is switched on (wfft_profile) each launch
// is bracketed by CUDA events on its own stream, and the kernel's algorithmic
// DRAM bytes and flops (compulsory traffic / arithmetic, not measured
// counters) are accumulated next to the measured time.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace wfft {

// Must match the WFFT_K_* constants of include/wfft.h.
enum KernelKind {
  KK_XFWD_PLAIN = 0, KK_XFWD_PUPD, KK_XFWD_RUPD, KK_XFWD_CONV,
  KK_XINV_APPLY, KK_XINV_RESID, KK_XINV_PREC, KK_XMID,
  KK_COL_FWD, KK_COL_INV, KK_COL_GRAD, KK_COL_DIV, KK_COL_PREC,
  KK_NEWMARK, KK_SCALAR, KK_NET_CONV, KK_NET_AUX, KK_XINV_PUPD, KK_NKIND
};

struct Profiler {
  bool on = false;
  long long launches[2][KK_NKIND] = {};
  long long lifetime = 0;  // every launch since creation (not reset by profiling)
  long long timed[2][KK_NKIND] = {};
  double ms[2][KK_NKIND] = {};
  double bytes[2][KK_NKIND] = {};
  double flops[2][KK_NKIND] = {};
  std::vector<cudaEvent_t> pool;
  int used = 0;
  struct Rec {
    int prec, kind, e0, e1;
    double bytes, flops;
  };
  std::vector<Rec> recs;

  int take() {
    if (used == (int)pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool.push_back(e);
    }
    return used++;
  }
  // fold the recorded launches into the totals (the stream must be idle)
  void collect() {
    for (const Rec& r : recs) {
      float t = 0.f;
      if (r.e0 >= 0 && r.e1 >= 0 && cudaEventElapsedTime(&t, pool[r.e0], pool[r.e1]) == cudaSuccess) {
        ms[r.prec][r.kind] += t;
        timed[r.prec][r.kind] += 1;
        bytes[r.prec][r.kind] += r.bytes;
        flops[r.prec][r.kind] += r.flops;
      }
    }
    recs.clear();
    used = 0;
  }
  void reset() {
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < KK_NKIND; ++k) launches[p][k] = timed[p][k] = 0, ms[p][k] = bytes[p][k] = flops[p][k] = 0;
    recs.clear();
    used = 0;
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// Profiler of the handle whose API call is running on this thread (or null).
extern thread_local Profiler* g_prof;

template <typename F>
inline void prof_launch(int prec, int kind, double bytes, double flops, cudaStream_t st, F&& launch) {
  Profiler* p = g_prof;
  if (!p) {
    launch();
    return;
  }
  p->launches[prec][kind] += 1;
  p->lifetime += 1;
  if (!p->on) {
    launch();
    return;
  }
  const int e0 = p->take(), e1 = p->take();
  if (e0 >= 0) cudaEventRecord(p->pool[e0], st);
  launch();
  if (e1 >= 0) cudaEventRecord(p->pool[e1], st);
  p->recs.push_back({prec, kind, e0, e1, bytes, flops});
}

}  // namespace wfft
