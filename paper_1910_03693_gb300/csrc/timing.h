// Per-launch instrumentation: a launch counter that is always kept, and,
// when enabled, a pair of CUDA events recorded on the launch stream around
// every kernel so that per-kernel device time can be read after a sync.  A
// selection of kernel names restricts the events to those kernels (the
// others are only counted): each event pair adds two stream operations around
// its kernel, so a step instrumented everywhere runs slower than the work it
// measures.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

struct fr_ctx;

namespace frgb {

struct TimerRec {
  const char* name;
  cudaEvent_t a, b;        // null for a launch that is only counted
  double bytes, flops;
};

struct TimerAcc {
  double ms = 0.0;
  long long count = 0;
  double bytes = 0.0;     // algorithmic bytes of all recorded launches
  double flops = 0.0;     // algorithmic floating-point operations of all recorded launches
};

struct Timing {
  bool on = false;
  bool capture = false;     // launches are being captured into a CUDA graph
  int64_t mark = 0;         // pending.size() when the current capture began
  long long launches = 0;
  std::vector<std::string> select;   // names whose launches get events (empty: all)
  int select_gen = 0;                // bumped on every change of the selection
  std::vector<cudaEvent_t> pool;
  std::vector<TimerRec> pending;
  std::map<std::string, TimerAcc> acc;
  cudaEvent_t take() {
    cudaEvent_t e;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  bool selected(const char* name) const {
    if (select.empty()) return true;
    for (const auto& n : select)
      if (n == name) return true;
    return false;
  }
  void give_back(const TimerRec& r) {
    if (r.a) pool.push_back(r.a);
    if (r.b) pool.push_back(r.b);
  }
  void add(const TimerRec& r) {
    float ms = 0.f;
    if (r.a) {
      cudaEventSynchronize(r.b);
      cudaEventElapsedTime(&ms, r.a, r.b);
    }
    auto& x = acc[r.name];
    x.ms += ms;
    x.count += 1;
    x.bytes += r.bytes;
    x.flops += r.flops;
  }
  void collect() {
    for (auto& r : pending) {
      add(r);
      give_back(r);
    }
    pending.clear();
  }
  // Accumulate the timers of one replay of a graph (the events belong to the graph).
  void accumulate(const std::vector<TimerRec>& recs) {
    for (const auto& r : recs) add(r);
  }
  ~Timing() {
    for (auto& r : pending) {
      if (r.a) cudaEventDestroy(r.a);
      if (r.b) cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

Timing& timing_of(fr_ctx* c);

// RAII scope around one kernel launch.
struct LaunchScope {
  Timing& t;
  const char* name;
  cudaStream_t s;
  double bytes, flops;
  cudaEvent_t a = nullptr;
  LaunchScope(fr_ctx* c, const char* n, cudaStream_t st, double b = 0.0, double f = 0.0)
      : t(timing_of(c)), name(n), s(st), bytes(b), flops(f) {
    ++t.launches;
    if (t.on && t.selected(n)) {
      a = t.take();
      record(a);
    }
  }
  // inside a stream capture the event becomes an event-record node of the graph
  void record(cudaEvent_t e) {
    if (t.capture) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
  }
  ~LaunchScope() {
    if (t.on) {
      cudaEvent_t b = nullptr;
      if (a) {
        b = t.take();
        record(b);
      }
      t.pending.push_back(TimerRec{name, a, b, bytes, flops});
    }
  }
};

}  // namespace frgb

#define FR_LAUNCH(ctx, name, stream, ...)                   \
  do {                                                      \
    ::frgb::LaunchScope _fr_scope((ctx), (name), (stream)); \
    __VA_ARGS__;                                            \
  } while (0)

// Same, recording `bytes` algorithmic bytes for the launch.
#define FR_LAUNCH_B(ctx, name, stream, bytes, ...)                               \
  do {                                                                           \
    ::frgb::LaunchScope _fr_scope((ctx), (name), (stream), (double)(bytes));     \
    __VA_ARGS__;                                                                 \
  } while (0)

// Same, recording algorithmic bytes and floating-point operations.
#define FR_LAUNCH_BF(ctx, name, stream, bytes, flops, ...)                                   \
  do {                                                                                       \
    ::frgb::LaunchScope _fr_scope((ctx), (name), (stream), (double)(bytes), (double)(flops)); \
    __VA_ARGS__;                                                                             \
  } while (0)

namespace frgb {
// Algorithmic operation counts of the FR operators as formulated (FMA = 2):
// per solution point of the volume residual, per face point of the traces,
// per mortar point of the common flux.
// diag: axis-aligned affine elements, whose metric products are one multiply
// per component.
inline double flops_volume(int nd, int P, bool visc, bool diag = false) {
  const int nv = nd + 2;
  double f = 1 + nd + 2 * nd + 3 + nd * (nd + 3);                  // inviscid flux
  f += diag ? nd * nv : nd * nv * 2 * nd;                            // transformed flux
  f += nd * nv * (2 * P + 4);                                        // divergence + correction
  f += 2 * nv;                                                       // -div / |J|
  if (visc) {
    f += nd * nv * (2 * P + 4);                                      // corrected gradient
    f += diag ? nd + nd * nv : nd * nv * (2 * nd + 1);               // physical gradient
    f += 2 + nd + 3 * nd * nd + 3 * nd + 2 * nd * nd + 2 * nd + (nd - 1) + 3 * nd * nd + 2 * nd * nd + 2 * nd;
    f += nd * nv;                                                    // f_inv - f_v
  }
  return f;
}
inline double flops_trace(int nd, int P, bool visc, bool diag = false) {
  const int nv = nd + 2;
  double f = nv * 2 * P;
  if (visc) f += nv * 2 * P * nd + (diag ? 2 * nd * nv : nd * nv * (2 * nd + 1));
  return f;
}
inline double flops_face(int nd, bool visc, bool diag = false) {
  const int nv = nd + 2;
  double f = 2 * (6 + 3 * nd + 3 * nd) + 1 + 6 * nv + 3 * nd + 2;   // two normal fluxes, Rusanov, area
  if (visc) {
    if (!diag) {
      const double fv = 2 + nd + 3 * nd * nd + 3 * nd + 2 * nd * nd + 2 * nd + (nd - 1) + 3 * nd * nd + 2 * nd * nd + 2 * nd;
      f += 2 * nv + 2 * (2 * nd + 1) + 8 * nd * nv + fv + 2 * nd * nv + nv + 4 * nv;
    } else {
      // lifting terms along the face axis only; one row of the viscous flux
      const double fr = 2 + nd + 3 * nd * nd + (nd - 1) + 2 * nd + 5 + 3 * nd + 2 * nd + 2;
      f += 2 * nv + 2 * (2 * nd + 1) + 2 * nd * nv + 6 * nv + fr + 2 * nv + nv + 4 * nv;
    }
  }
  return f;
}
// Algorithmic data movement (values; times the operand size gives bytes):
// what each kernel has to read and write at least, geometry excluded.
// Traces, per element: the state in, every face's q (and for NS the gradient) out.
inline double values_trace(int nd, int P, bool visc) {
  const int nv = nd + 2, nsp = nd == 2 ? P * P : P * P * P, nfp = nd == 2 ? P : P * P;
  return (double)nv * nsp + 2.0 * nd * nfp * (visc ? nv * (1 + nd) : nv);
}
// Volume kernel, per element: the state (and the tangent), the face outputs it
// reads (common flux; for NS also q^com - q; the JVP's tangents of both), and
// the result, in units of the operand size except the result (out_ratio =
// result size / operand size, 2 for an FP64 result of FP32 kernels).
inline double values_volume(int nd, int P, bool visc, bool jvp, double out_ratio = 1.0) {
  const int nv = nd + 2, nsp = nd == 2 ? P * P : P * P * P, nfp = nd == 2 ? P : P * P;
  const double in = (double)nv * nsp * (jvp ? 2 : 1) + 2.0 * nd * nfp * nv * (visc ? (jvp ? 3 : 2) : 1);
  return in + out_ratio * nv * nsp;
}
// Interior face kernel, per mortar point (conforming faces): both sides'
// traces (and tangent traces) in, both sides' outputs out.
inline double values_face(int nd, bool visc, bool jvp) {
  const int nv = nd + 2;
  const double in = 2.0 * (visc ? nv * (1 + nd) : nv) * (jvp ? 2 : 1);
  const double out = 2.0 * nv * (visc ? (jvp ? 3 : 2) : 1);
  return in + out;
}
}  // namespace frgb
