// Matrix-free Newton-Krylov of Sec. 2.3: restarted GMRES(m) on
// (sigma I - dR/dq) dq = F with FP64 Arnoldi (classical Gram-Schmidt, once or
// with re-orthogonalisation; Givens rotations), and one ESDIRK stage by pseudo-transient
// continuation with the SER pseudo-time step and dtau back-off.
//
// Reductions are deterministic: every block writes its partial sums to a
// fixed slot and the last block to finish adds the slots in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fr_launch.h"

namespace frgb {

constexpr int kRedBlocks = 608;     // most blocks of a reduction: 4 per SM on 152 SMs (grid-stride)
constexpr int kRedThreads = 256;
constexpr int kMaxK = 64;           // most vectors in one multi-dot (restart length + 1)

// reduction scratch (doubles): per-block partials [kRedBlocks][kMaxK], then the
// reduced values H1 (first Gram-Schmidt pass, ||w||^2 after the dots), H2
// (second pass), N (||w||^2 after an update), Y (the GMRES coefficients), S
// (the scales of the stored Krylov columns) and one slot holding the arrival
// counter of the grid reductions
constexpr int64_t kOutH1 = (int64_t)kRedBlocks * kMaxK;
constexpr int64_t kOutH2 = kOutH1 + kMaxK;
constexpr int64_t kOutN = kOutH2 + kMaxK;
constexpr int64_t kOutY = kOutN + kMaxK;
constexpr int64_t kOutS = kOutY + kMaxK;    // scales of the stored Krylov columns
constexpr int64_t kTicket = kOutS + kMaxK;

// State of a device-driven GMRES cycle (doubles of fr_ctx::d_gm): the
// Hessenberg columns (column j at j * kMaxK, rows 0..j+1, rotated in place),
// the Givens rotations, the right-hand side g of the small least-squares
// problem, then the control words (ints): the gate, the iterations completed
// in the cycle, and a flag set when an Arnoldi vector was not finite.
constexpr int64_t kGmH = 0;
constexpr int64_t kGmCs = kGmH + (int64_t)kMaxK * kMaxK;
constexpr int64_t kGmSn = kGmCs + kMaxK;
constexpr int64_t kGmG = kGmSn + kMaxK;
constexpr int64_t kGmCtl = kGmG + kMaxK + 1;
constexpr int64_t kGmSize = kGmCtl + 2;

static fr_status ensure_red(fr_ctx* c) {
  if (c->d_red) return FR_OK;
  c->red_cap = kTicket + 1;
  if (cudaMalloc(&c->d_red, sizeof(double) * c->red_cap) != cudaSuccess) return FR_ERR_NOMEM;
  if (cudaMemset(c->d_red, 0, sizeof(double) * c->red_cap) != cudaSuccess) return FR_ERR_CUDA;
  // host mirror: H1, H2, N (read back), then the column scales (uploaded)
  if (cudaMallocHost(&c->h_red, sizeof(double) * 4 * kMaxK) != cudaSuccess) return FR_ERR_NOMEM;
  return FR_OK;
}

static unsigned* ticket_of(fr_ctx* c) { return reinterpret_cast<unsigned*>(c->d_red + kTicket); }

// Blocks of a reduction over n values: enough to fill every SM, no more than
// one pair of values per thread.
static unsigned red_blocks(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + 2 * kRedThreads - 1) / (2 * kRedThreads)));
}

// Sum vals[0..k) over the grid into out[0..k), deterministically: every block
// writes its sums (warp-shuffle then shared-memory tree, fixed order) to its
// own slot of `partial`; the last block to arrive (arrival counter) adds the
// slots in a fixed order, writes out[] and re-arms the counter.
// Returns true in the block that wrote out[] (after its threads < k stored it).
template <int KC>
__device__ __forceinline__ bool grid_sum(const double (&vals)[KC], int k, double* __restrict__ partial,
                                         double* __restrict__ out, unsigned* __restrict__ ticket) {
  __shared__ double red[kRedThreads / 32][KC];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) {
    if (kk < k) {
      double v = vals[kk];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][kk] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double t = 0.0;
#pragma unroll
    for (int wi = 0; wi < kRedThreads / 32; ++wi) t += red[wi][threadIdx.x];
    partial[(int64_t)blockIdx.x * kMaxK + threadIdx.x] = t;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // the last block: thread t adds the slots t, t + blockDim, ... (all loads of
  // a thread issued together), then the same warp/shared-memory tree as above
  constexpr int kSlots = (kRedBlocks + kRedThreads - 1) / kRedThreads;
  double tot[KC];
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) tot[kk] = 0.0;
#pragma unroll
  for (int r = 0; r < kSlots; ++r) {
    const int bl = threadIdx.x + r * kRedThreads;
    if (bl < (int)gridDim.x) {
#pragma unroll
      for (int kk = 0; kk < KC; ++kk)
        if (kk < k) tot[kk] += __ldcg(partial + (int64_t)bl * kMaxK + kk);
    }
  }
  __syncthreads();
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) {
    if (kk < k) {
      double v = tot[kk];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][kk] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double t = 0.0;
#pragma unroll
    for (int wi = 0; wi < kRedThreads / 32; ++wi) t += red[wi][threadIdx.x];
    out[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Bookkeeping of Arnoldi iteration j in a device-driven GMRES cycle, run by
// the block that completes the iteration's last Gram-Schmidt update: column j
// of the Hessenberg matrix of the operator (h_ij = s_i raw_ij from the
// coefficients of the unnormalised basis, plus the second pass's, plus the
// shift on the diagonal, h_{j+1,j} = ||w_new||), the earlier Givens rotations
// applied to it, the new rotation and the least-squares residual estimate
// |g_{j+1}|.  The gate closes when that estimate reaches tol, when the new
// vector is zero (the Krylov space is invariant), after the iteration limit
// (last) or when ||w_new|| is not finite (then ctl[2] = 1 and the column is
// not counted); ctl[1] counts the iterations of the cycle that completed.
// The column and the rotations are staged in shared memory so that the one
// thread applying the rotations in order waits on no global load.
struct StepArgs {
  double* gm = nullptr;              // cycle state (kGm* layout); null: no step after this pass
  const double* dots1 = nullptr;     // the Gram-Schmidt coefficients of the pass(es)
  const double* dots2 = nullptr;
  const double* scale = nullptr;     // scales of the stored columns
  const double* nrm2 = nullptr;      // ||w_new||^2
  double shift = 0.0, tol = 0.0;
  int j = 0, last = 0, two_pass = 0;
};

__device__ void arnoldi_step_block(const StepArgs& a) {
  __shared__ double col[kMaxK + 1], rc[kMaxK], rs[kMaxK];
  __shared__ int keep;
  double* gm = a.gm;
  int* ctl = reinterpret_cast<int*>(gm + kGmCtl);
  const int j = a.j;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double h1 = a.scale[i] * a.dots1[i];
    col[i] = a.two_pass ? h1 + a.scale[i] * a.dots2[i] : h1;
    if (i < j) {
      rc[i] = gm[kGmCs + i];
      rs[i] = gm[kGmSn + i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = sqrt(*a.nrm2);
    keep = isfinite(hn) ? 1 : 0;
    if (!keep) {
      ctl[2] = 1;
      ctl[0] = 1;
    } else {
      col[j] += a.shift;
      col[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = rc[i] * col[i] + rs[i] * col[i + 1];
        col[i + 1] = -rs[i] * col[i] + rc[i] * col[i + 1];
        col[i] = t;
      }
      const double den = hypot(col[j], col[j + 1]);
      const double rcj = den == 0.0 ? 1.0 : col[j] / den;
      const double sj = den == 0.0 ? 0.0 : col[j + 1] / den;
      col[j] = rcj * col[j] + sj * col[j + 1];
      col[j + 1] = 0.0;
      gm[kGmCs + j] = rcj;
      gm[kGmSn + j] = sj;
      const double gj = gm[kGmG + j];
      gm[kGmG + j + 1] = -sj * gj;
      gm[kGmG + j] = rcj * gj;
      ctl[1] = j + 1;
      if (fabs(sj * gj) <= a.tol || hn == 0.0 || a.last) ctl[0] = 1;
    }
  }
  __syncthreads();
  if (keep)
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) gm[kGmH + (int64_t)j * kMaxK + i] = col[i];
}

// Slot q of a vector seen as pairs (VEC: 16-byte loads of two values) or
// single values: slot nw = n / W is the odd tail (one value) when VEC and n is
// odd; slots beyond the vector read as zero.
template <bool VEC>
struct Slots {
  static constexpr int W = VEC ? 2 : 1;
  // streaming load (the Krylov columns: read once per pass)
  __device__ static void load_stream(const double* __restrict__ p, int64_t q, int64_t nw, int64_t n, double (&x)[2]) {
    if (q < nw) {
      if (VEC) {
        const double2 t = __ldcs(reinterpret_cast<const double2*>(p + 2 * q));
        x[0] = t.x;
        x[1] = t.y;
      } else {
        x[0] = __ldcs(p + q);
        x[1] = 0.0;
      }
    } else {
      x[0] = (VEC && q == nw && (n & 1)) ? p[2 * nw] : 0.0;
      x[1] = 0.0;
    }
  }
  // ordinary load (w: read again by the update that follows)
  __device__ static void load(const double* __restrict__ p, int64_t q, int64_t nw, int64_t n, double (&x)[2]) {
    if (q < nw) {
      if (VEC) {
        const double2 t = *reinterpret_cast<const double2*>(p + 2 * q);
        x[0] = t.x;
        x[1] = t.y;
      } else {
        x[0] = p[q];
        x[1] = 0.0;
      }
    } else {
      x[0] = (VEC && q == nw && (n & 1)) ? p[2 * nw] : 0.0;
      x[1] = 0.0;
    }
  }
  __device__ static void store(double* __restrict__ p, int64_t q, int64_t nw, int64_t n, const double (&x)[2]) {
    if (q < nw) {
      if (VEC) *reinterpret_cast<double2*>(p + 2 * q) = make_double2(x[0], x[1]);
      else p[q] = x[0];
    } else if (VEC && q == nw && (n & 1)) {
      p[2 * nw] = x[0];
    }
  }
};

// Slots handled per thread and loop step: U slots spaced one grid apart, all
// their loads issued before any arithmetic (bytes in flight per thread scale
// with U), fewer for many columns to bound the registers.
template <int KC, int MAP = 0>
struct Unroll {
  // MAP 0: U slots a thread spaced one grid apart; MAP 1 (the default): every
  // warp reads U consecutive 32-slot runs of each column (U x 512 bytes
  // contiguous a column), four slots and four columns a load batch.  Measured
  // at 32^3 (30 Arnoldi iterations): dots 2.9 -> 4.2 TB/s, updates 4.0 -> 4.4
  // TB/s; reading many columns at once, DRAM serves long runs of each column
  // better than single 512-byte segments spread over the whole vector
  static constexpr int U = MAP == 1 ? 4 : (KC <= 2 ? 4 : (KC <= 8 ? 2 : 1));
  static constexpr int CH = MAP == 1 ? (KC < 4 ? KC : 4) : (KC < 8 ? KC : 8);   // columns per load batch
  // accumulators per column: more than one breaks the FMA dependence chain
  // but costs registers and occupancy, and measured slower in the solver
  static constexpr int A = 1;
};

// Slot q of the vector w as FP64 values: w is FP64, or the FP32 output of the
// JVP (converted); NEG negates it (w = -J v), which costs nothing in the FMAs.
template <bool VEC, typename WT, bool NEG>
struct WSlots {
  __device__ static void load(const WT* p, int64_t q, int64_t nw, int64_t n, double (&x)[2]) {
    if (q < nw) {
      if (VEC) {
        if constexpr (sizeof(WT) == 8) {
          const double2 t = *reinterpret_cast<const double2*>(p + 2 * q);
          x[0] = t.x;
          x[1] = t.y;
        } else {
          const float2 t = *reinterpret_cast<const float2*>(p + 2 * q);
          x[0] = (double)t.x;
          x[1] = (double)t.y;
        }
      } else {
        x[0] = (double)p[q];
        x[1] = 0.0;
      }
    } else {
      x[0] = (VEC && q == nw && (n & 1)) ? (double)p[2 * nw] : 0.0;
      x[1] = 0.0;
    }
    if (NEG) {
      x[0] = -x[0];
      x[1] = -x[1];
    }
  }
};

// out[kk] = V[kk]^T w for kk < k, and, when with_norm, out[k] = ||w||^2.
// V == nullptr: out[0] = ||w||^2 alone.  V holds the stored (unscaled)
// Krylov columns; the caller applies their scales to the dots.
// Slot walk of the reduction kernels: the first slot of a thread, the
// distance between its U unrolled slots and the loop step.  MAP 0: slots one
// grid apart; MAP 1: each warp reads a run of U x 32 consecutive slots (the
// U loads of a lane one warp width apart), runs one grid of warps apart.
template <int MAP, int U>
struct SlotWalk {
  int64_t first, du, step;
  __device__ SlotWalk(int64_t stride) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (MAP == 1) {
      first = (g >> 5) * (U * 32) + (g & 31);
      du = 32;
      step = (stride >> 5) * (U * 32);
    } else {
      first = g;
      du = stride;
      step = U * stride;
    }
  }
};

template <int KC, bool VEC, typename WT, bool NEG, int MAP = 0>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const double* __restrict__ V, int64_t ldv, int k,
                                                           const WT* __restrict__ w, int64_t n,
                                                           double* __restrict__ partial, double* __restrict__ out,
                                                           unsigned* __restrict__ ticket, int with_norm,
                                                           const int* __restrict__ gate) {
  if (gate && *gate) return;   // past the end of a device-driven GMRES cycle
  constexpr int U = Unroll<KC, MAP>::U, CH = Unroll<KC, MAP>::CH;
  using L = Slots<VEC>;
  using LW = WSlots<VEC, WT, NEG>;
  constexpr int A = Unroll<KC>::A;
  double acc[A][KC + 1];
#pragma unroll
  for (int a = 0; a < A; ++a)
#pragma unroll
    for (int kk = 0; kk <= KC; ++kk) acc[a][kk] = 0.0;
  const int64_t nw = n / L::W, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t last = nw + ((VEC && (n & 1)) ? 0 : -1);   // highest slot holding data
  const SlotWalk<MAP, U> sw(stride);
  for (int64_t q0 = sw.first; q0 - (MAP == 1 ? (threadIdx.x & 31) : 0) <= last; q0 += sw.step) {
    double wv[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u) LW::load(w, q0 + u * sw.du, nw, n, wv[u]);
    if (V) {
#pragma unroll
      for (int c0 = 0; c0 < KC; c0 += CH) {
        if (c0 < k) {
          double vv[U][CH][2];
#pragma unroll
          for (int t = 0; t < CH; ++t)
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (c0 + t < k) L::load_stream(V + (c0 + t) * ldv, q0 + u * sw.du, nw, n, vv[u][t]);
#pragma unroll
          for (int t = 0; t < CH; ++t)
            if (c0 + t < k) {
#pragma unroll
              for (int u = 0; u < U; ++u)   // explicit FMA chain: one FP64 op per product
                acc[u % A][c0 + t] = fma(vv[u][t][1], wv[u][1], fma(vv[u][t][0], wv[u][0], acc[u % A][c0 + t]));
            }
        }
      }
    }
    // ||w||^2 only when asked for: on GB300 every FP64 FMA here costs about as
    // much time as the 8 bytes it is paired with
    if (!V || with_norm) {
#pragma unroll
      for (int u = 0; u < U; ++u) acc[u % A][KC] = fma(wv[u][1], wv[u][1], fma(wv[u][0], wv[u][0], acc[u % A][KC]));
    }
  }
  // fixed-order combination of the partial accumulators
#pragma unroll
  for (int a = 1; a < A; ++a)
#pragma unroll
    for (int kk = 0; kk <= KC; ++kk) acc[0][kk] += acc[a][kk];
  if (!V) {
    const double one[1] = {acc[0][KC]};
    grid_sum<1>(one, 1, partial, out, ticket);
    return;
  }
  // slots 0..k-1: the dots; slot k: ||w||^2 (selects only, no runtime indexing)
  double o[KC + 1];
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) o[kk] = kk < k ? acc[0][kk] : acc[0][KC];
  o[KC] = acc[0][KC];
  grid_sum<KC + 1>(o, with_norm ? k + 1 : k, partial, out, ticket);
}

// ---------------------------------------------------------------------------
// Double-float dot products of the Arnoldi process.  On GB300 the FP64 pipe
// issues 2 FMAs a clock per SM while HBM delivers about 2.7 values a clock per
// SM, so a dot product with one FP64 FMA per value cannot reach the memory
// bound.  Here every FP64 value is split into two FP32 numbers by integer
// operations on its bit pattern, and the products are accumulated as
// double-float sums (error-free transformations on the FP32 pipe: the exact
// product of the high parts through the FMA, the two cross terms, Knuth's
// TwoSum and Dekker's Fast2Sum); each thread's sum is converted to FP64 once,
// and the grid reduction stays FP64.
// ---------------------------------------------------------------------------

// x = hi + lo: hi holds x's leading 24 significant bits (truncated), lo the
// FP32 rounding of the exact remainder (its 29 trailing bits), so that
// |x - hi - lo| <= 2^-48 |x| for |x| >= 2^-83 (below, the remainder falls into
// FP32's subnormal range: absolute error under 2^-149).  Built from the bit
// pattern by integer operations, an int-to-float conversion and exact
// power-of-two scalings: no FP64 instruction.  |x| < 2^-126 gives (0, 0);
// |x| >= 2^128 gives the FP32 rounding of x.
__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int e = (int)((hw >> 20) & 0x7FF);
  const unsigned sign = hw & 0x80000000u;
  if (e < 897) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  if (e > 1150) {
    hi = __double2float_rn(x);
    lo = 0.0f;
    return;
  }
  hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  // remainder m29 2^(e - 1075), scaled in two exact steps that stay in range
  // (2^(e - 1011) then 2^-64, or 2^(e - 1139) then 2^64)
  const float m = __uint2float_rn(lw & 0x1FFFFFFFu);
  float r;
  if (e <= 1100) r = __fmul_rn(__fmul_rn(m, __uint_as_float((unsigned)(e - 1011 + 127) << 23)), __uint_as_float(63u << 23));
  else r = __fmul_rn(__fmul_rn(m, __uint_as_float((unsigned)(e - 1139 + 127) << 23)), __uint_as_float(191u << 23));
  lo = sign ? -r : r;
}

// (S, E) += a * b, a = (ah, al), b = (bh, bl): the exact product of the high
// parts and the two cross terms (the product of the low parts, 2^-46 of ab,
// is dropped), added with TwoSum and renormalised with Fast2Sum
__device__ __forceinline__ void df_madd(float& S, float& E, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  const float s = __fadd_rn(S, p);
  const float bb = __fsub_rn(s, S);
  const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float u = __fadd_rn(t, __fadd_rn(E, pe));
  S = __fadd_rn(s, u);
  E = __fsub_rn(u, __fsub_rn(S, s));
}

// out[kk] = V[kk]^T w for kk < k (and ||w||^2 with with_norm), as k_multidot,
// accumulated in double-float arithmetic.  w is FP64 (WT, NEG as k_multidot,
// only double / false are instantiated).
template <int KC, bool VEC, typename WT, bool NEG, int MAP = 0>
__global__ void __launch_bounds__(kRedThreads) k_multidot_df(const double* __restrict__ V, int64_t ldv, int k,
                                                              const WT* __restrict__ w, int64_t n,
                                                              double* __restrict__ partial, double* __restrict__ out,
                                                              unsigned* __restrict__ ticket, int with_norm,
                                                              const int* __restrict__ gate) {
  static_assert(sizeof(WT) == 8 && !NEG, "FP64 vectors only");
  if (gate && *gate) return;
  constexpr int U = Unroll<KC>::U, CH = Unroll<KC>::CH;
  using L = Slots<VEC>;
  float S[KC + 1], E[KC + 1];
#pragma unroll
  for (int kk = 0; kk <= KC; ++kk) S[kk] = E[kk] = 0.0f;
  const int64_t nw = n / L::W, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t last = nw + ((VEC && (n & 1)) ? 0 : -1);
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q0 <= last; q0 += U * stride) {
    double wv[U][2];
    float wh[U][2], wl[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      L::load(w, q0 + u * stride, nw, n, wv[u]);
      split_df(wv[u][0], wh[u][0], wl[u][0]);
      split_df(wv[u][1], wh[u][1], wl[u][1]);
    }
#pragma unroll
    for (int c0 = 0; c0 < KC; c0 += CH) {
      if (c0 < k) {
        double vv[U][CH][2];
#pragma unroll
        for (int t = 0; t < CH; ++t)
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (c0 + t < k) L::load_stream(V + (c0 + t) * ldv, q0 + u * stride, nw, n, vv[u][t]);
#pragma unroll
        for (int t = 0; t < CH; ++t)
          if (c0 + t < k) {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                float vh, vl;
                split_df(vv[u][t][h], vh, vl);
                df_madd(S[c0 + t], E[c0 + t], vh, vl, wh[u][h], wl[u][h]);
              }
          }
      }
    }
    if (with_norm) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) df_madd(S[KC], E[KC], wh[u][h], wl[u][h], wh[u][h], wl[u][h]);
    }
  }
  double o[KC + 1];
#pragma unroll
  for (int kk = 0; kk <= KC; ++kk) o[kk] = (double)S[kk] + (double)E[kk];
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) o[kk] = kk < k ? o[kk] : o[KC];
  grid_sum<KC + 1>(o, with_norm ? k + 1 : k, partial, out, ticket);
}

// w_out = w_in - sum_kk s_kk^2 raw[kk] V[kk] (the stored columns V[kk] scaled
// by s_kk are the orthonormal basis, raw[kk] = V[kk]^T w_in); out[0] =
// ||w_out||^2.  w_out may be w_in (in place, FP64).  With next_scale, the
// block that finishes the norm also stores 1/||w_out|| there (0 for a zero
// vector) and next_j into *jidx: the scale and index of the next Arnoldi
// product, set without a round trip through the host (the host computes the
// same IEEE quotient for its own copy).
template <int KC, bool VEC, typename WT, bool NEG, int MAP = 0>
__global__ void __launch_bounds__(kRedThreads) k_orth_update(const double* __restrict__ V, int64_t ldv, int k,
                                                              const double* __restrict__ raw,
                                                              const double* __restrict__ scale, const WT* w_in,
                                                              double* w_out, int64_t n, double* __restrict__ partial,
                                                              double* __restrict__ out, unsigned* __restrict__ ticket,
                                                              double* __restrict__ next_scale, int* __restrict__ jidx,
                                                              int next_j, const int* __restrict__ gate, StepArgs step) {
  if (gate && *gate) return;
  constexpr int U = Unroll<KC, MAP>::U, CH = Unroll<KC, MAP>::CH;
  using L = Slots<VEC>;
  using LW = WSlots<VEC, WT, NEG>;
  __shared__ double hs[KC];
  if (threadIdx.x < KC) hs[threadIdx.x] = threadIdx.x < k ? scale[threadIdx.x] * scale[threadIdx.x] * raw[threadIdx.x] : 0.0;
  __syncthreads();
  double accu[U] = {};
  const int64_t nw = n / L::W, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t last = nw + ((VEC && (n & 1)) ? 0 : -1);
  const SlotWalk<MAP, U> sw(stride);
  for (int64_t q0 = sw.first; q0 - (MAP == 1 ? (threadIdx.x & 31) : 0) <= last; q0 += sw.step) {
    double x[U][2];
#pragma unroll
    for (int u = 0; u < U; ++u) LW::load(w_in, q0 + u * sw.du, nw, n, x[u]);
#pragma unroll
    for (int c0 = 0; c0 < KC; c0 += CH) {
      if (c0 < k) {
        double vv[U][CH][2];
#pragma unroll
        for (int t = 0; t < CH; ++t)
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (c0 + t < k) L::load_stream(V + (c0 + t) * ldv, q0 + u * sw.du, nw, n, vv[u][t]);
#pragma unroll
        for (int t = 0; t < CH; ++t)
          if (c0 + t < k) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              x[u][0] -= hs[c0 + t] * vv[u][t][0];
              x[u][1] -= hs[c0 + t] * vv[u][t][1];
            }
          }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      L::store(w_out, q0 + u * sw.du, nw, n, x[u]);
      accu[u] = fma(x[u][1], x[u][1], fma(x[u][0], x[u][0], accu[u]));
    }
  }
  double acc[1] = {accu[0]};
#pragma unroll
  for (int u = 1; u < U; ++u) acc[0] += accu[u];
  if (grid_sum<1>(acc, 1, partial, out, ticket)) {   // the block that completed the sum
    if (threadIdx.x == 0 && next_scale) {
      const double hn = sqrt(out[0]);
      *next_scale = hn != 0.0 ? 1.0 / hn : 0.0;
      *jidx = next_j;
    }
    if (step.gm) arnoldi_step_block(step);
  }
}

// Blocks of one reduction launch: at most `grid`, and no more than the SMs
// hold at once for this kernel (its register count decides), so that the
// grid-stride loop runs as whole waves; the occupancy query runs once per
// kernel instantiation.
template <auto KERN>
static unsigned wave_grid(unsigned grid) {
  static int resident = 0;
  if (resident == 0) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, KERN, kRedThreads, 0) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    resident = std::max(1, per_sm * std::max(sms, 1));
  }
  return std::max(1u, std::min(grid, (unsigned)resident));
}

// ---------------------------------------------------------------------------
// Krylov basis stored in FP32 (GMRES with FP32 products and a tolerance those
// products can meet).  The columns and the product J v are FP32, so every
// Arnoldi kernel moves 4 bytes a value where the FP64 basis moves 8.  The
// arithmetic must leave the FP64 pipe for that to pay: on GB300 one FP64 FMA
// per value already runs at about the rate HBM delivers 8-byte values.  Each
// thread therefore sums its 16 products of a loop step (four float4 slots a
// column) with FP32 FMAs and adds that partial sum to an FP64 accumulator, one
// FP64 addition per 16 values and column, before the usual deterministic FP64
// grid reduction.  A partial sum carries a relative error of about 16 x 2^-24
// of its sixteen |u_i w_i|: the dots, norms and hence the orthogonality of the
// stored basis hold to about 1e-6, the accuracy of the FP32 products
// themselves.  Compressed-basis GMRES (Aliaga, Anzt, Gruetzmacher,
// Quintana-Orti, Tomas, IJHPCA 2022) stores the basis in reduced precision for
// the same reason.
// ---------------------------------------------------------------------------

// Slot q of an FP32 vector of n values as four values; the slot n / 4 holds
// the ragged tail, slots past the vector read as zero.
struct F4Slots {
  __device__ static float4 tail(const float* p, int64_t n4, int64_t n) {
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t b = 4 * n4;
    if (b < n) r.x = p[b];
    if (b + 1 < n) r.y = p[b + 1];
    if (b + 2 < n) r.z = p[b + 2];
    return r;
  }
  // streaming load (the Krylov columns: read once per pass)
  __device__ static float4 load_stream(const float* __restrict__ p, int64_t q, int64_t n4, int64_t n) {
    if (q < n4) return __ldcs(reinterpret_cast<const float4*>(p) + q);
    return q == n4 ? tail(p, n4, n) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ static float4 load(const float* p, int64_t q, int64_t n4, int64_t n) {
    if (q < n4) return reinterpret_cast<const float4*>(p)[q];
    return q == n4 ? tail(p, n4, n) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ static void store(float* p, int64_t q, int64_t n4, int64_t n, float4 v) {
    if (q < n4) {
      reinterpret_cast<float4*>(p)[q] = v;
    } else if (q == n4) {
      const int64_t b = 4 * n4;
      if (b < n) p[b] = v.x;
      if (b + 1 < n) p[b + 1] = v.y;
      if (b + 2 < n) p[b + 2] = v.z;
    }
  }
};

__device__ __forceinline__ float dot4(float4 a, float4 b, float s) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
}

// out[kk] = s_w V[kk]^T w for kk < k (s_w = -1 with NEG: w holds J v and the
// Arnoldi vector is -J v), and with with_norm out[k] = ||w||^2; FP32 columns
// and w, walked as warp runs of U x 32 float4 slots.
template <int KC, bool NEG>
__global__ void __launch_bounds__(kRedThreads) k_multidot32(const float* __restrict__ V, int64_t ldv, int k,
                                                             const float* __restrict__ w, int64_t n,
                                                             double* __restrict__ partial, double* __restrict__ out,
                                                             unsigned* __restrict__ ticket, int with_norm,
                                                             const int* __restrict__ gate) {
  if (gate && *gate) return;
  // two columns a load batch: 32 registers of column values in flight, so
  // that two CTAs of 256 threads fit on an SM up to KC = 8
  constexpr int U = 4, CH = KC < 2 ? KC : 2;
  double acc[KC + 1];
#pragma unroll
  for (int kk = 0; kk <= KC; ++kk) acc[kk] = 0.0;
  const int64_t n4 = n / 4, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t last = n4 + ((n & 3) ? 0 : -1);   // highest slot holding data
  const SlotWalk<1, U> sw(stride);
  for (int64_t q0 = sw.first; q0 - (threadIdx.x & 31) <= last; q0 += sw.step) {
    float4 wv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) wv[u] = F4Slots::load(w, q0 + u * sw.du, n4, n);
#pragma unroll
    for (int c0 = 0; c0 < KC; c0 += CH) {
      if (c0 < k) {
        float4 vv[U][CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (c0 + t < k) vv[u][t] = F4Slots::load_stream(V + (c0 + t) * ldv, q0 + u * sw.du, n4, n);
#pragma unroll
        for (int t = 0; t < CH; ++t)
          if (c0 + t < k) {
            float sp = 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) sp = dot4(vv[u][t], wv[u], sp);
            acc[c0 + t] += (double)sp;
          }
      }
    }
    if (with_norm) {
      float sp = 0.f;
#pragma unroll
      for (int u = 0; u < U; ++u) sp = dot4(wv[u], wv[u], sp);
      acc[KC] += (double)sp;
    }
  }
  // slots 0..k-1: the dots; slot k: ||w||^2 (selects only, no runtime indexing)
  double o[KC + 1];
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) o[kk] = kk < k ? (NEG ? -acc[kk] : acc[kk]) : acc[KC];
  o[KC] = acc[KC];
  grid_sum<KC + 1>(o, with_norm ? k + 1 : k, partial, out, ticket);
}

// w_out = s_w w_in - sum_kk s_kk^2 raw[kk] V[kk] in FP32 (s_w = -1 with NEG),
// out[0] = ||w_out||^2; w_out may be w_in.  With next_scale, the block that
// finishes the norm stores 1/||w_out|| and next_j as k_orth_update does.
template <int KC, bool NEG>
__global__ void __launch_bounds__(kRedThreads) k_orth_update32(const float* __restrict__ V, int64_t ldv, int k,
                                                                const double* __restrict__ raw,
                                                                const double* __restrict__ scale, const float* w_in,
                                                                float* w_out, int64_t n, double* __restrict__ partial,
                                                                double* __restrict__ out, unsigned* __restrict__ ticket,
                                                                double* __restrict__ next_scale, int* __restrict__ jidx,
                                                                int next_j, const int* __restrict__ gate, StepArgs step) {
  if (gate && *gate) return;
  constexpr int U = 4, CH = KC < 4 ? KC : 4;
  __shared__ float hs[KC];
  if (threadIdx.x < KC)
    hs[threadIdx.x] = threadIdx.x < k ? (float)(scale[threadIdx.x] * scale[threadIdx.x] * raw[threadIdx.x]) : 0.f;
  __syncthreads();
  double accn = 0.0;
  const int64_t n4 = n / 4, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t last = n4 + ((n & 3) ? 0 : -1);
  const SlotWalk<1, U> sw(stride);
  for (int64_t q0 = sw.first; q0 - (threadIdx.x & 31) <= last; q0 += sw.step) {
    float4 x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      x[u] = F4Slots::load(w_in, q0 + u * sw.du, n4, n);
      if (NEG) x[u] = make_float4(-x[u].x, -x[u].y, -x[u].z, -x[u].w);
    }
#pragma unroll
    for (int c0 = 0; c0 < KC; c0 += CH) {
      if (c0 < k) {
        float4 vv[U][CH];
#pragma unroll
        for (int t = 0; t < CH; ++t)
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (c0 + t < k) vv[u][t] = F4Slots::load_stream(V + (c0 + t) * ldv, q0 + u * sw.du, n4, n);
#pragma unroll
        for (int t = 0; t < CH; ++t)
          if (c0 + t < k) {
            const float h = -hs[c0 + t];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              x[u].x = fmaf(h, vv[u][t].x, x[u].x);
              x[u].y = fmaf(h, vv[u][t].y, x[u].y);
              x[u].z = fmaf(h, vv[u][t].z, x[u].z);
              x[u].w = fmaf(h, vv[u][t].w, x[u].w);
            }
          }
      }
    }
    float sp = 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      F4Slots::store(w_out, q0 + u * sw.du, n4, n, x[u]);
      sp = dot4(x[u], x[u], sp);
    }
    accn += (double)sp;
  }
  const double acc[1] = {accn};
  if (grid_sum<1>(acc, 1, partial, out, ticket)) {   // the block that completed the sum
    if (threadIdx.x == 0 && next_scale) {
      const double hn = sqrt(out[0]);
      *next_scale = hn != 0.0 ? 1.0 / hn : 0.0;
      *jidx = next_j;
    }
    if (step.gm) arnoldi_step_block(step);
  }
}

// x (+)= sum_kk y[kk] V[kk] with FP32 columns: the column sum in FP32, one
// FP64 addition a value (x is the FP64 Newton correction); accumulate 0 writes x
__global__ void k_combine32(const float* __restrict__ V, int64_t ldv, int k, const double* __restrict__ y,
                            double* __restrict__ x, int64_t n, int accumulate) {
  __shared__ float ys[kMaxK];
  if (threadIdx.x < k) ys[threadIdx.x] = (float)y[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float sp = 0.f;
    for (int kk = 0; kk < k; ++kk) sp = fmaf(ys[kk], V[kk * ldv + i], sp);
    x[i] = accumulate ? x[i] + (double)sp : (double)sp;
  }
}

// y = (float)(a x): the first Krylov column from the FP64 residual
__global__ void k_scale32(const double* __restrict__ x, double a, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)(a * x[i]);
}

// launch KERNEL<KC, VEC, WT, NEG> with the smallest KC >= k; VEC when every
// vector starts on a 16-byte boundary and the column stride is even
#define FR_KC_LAUNCH(KC_, V_, grid, KERNEL, WT, NEG, ...)                                                \
  do {                                                                                                  \
    if (c->arnoldi_map == 1)                                                                            \
      KERNEL<KC_, V_, WT, NEG, 1><<<wave_grid<KERNEL<KC_, V_, WT, NEG, 1>>(grid), kRedThreads, 0, s>>>(__VA_ARGS__); \
    else                                                                                                \
      KERNEL<KC_, V_, WT, NEG, 0><<<wave_grid<KERNEL<KC_, V_, WT, NEG, 0>>(grid), kRedThreads, 0, s>>>(__VA_ARGS__); \
  } while (0)
#define FR_KC_CASES(k, V_, grid, KERNEL, WT, NEG, ...)                                                   \
  do {                                                                                                  \
    if ((k) <= 1) FR_KC_LAUNCH(1, V_, grid, KERNEL, WT, NEG, __VA_ARGS__);                              \
    else if ((k) <= 2) FR_KC_LAUNCH(2, V_, grid, KERNEL, WT, NEG, __VA_ARGS__);                         \
    else if ((k) <= 4) FR_KC_LAUNCH(4, V_, grid, KERNEL, WT, NEG, __VA_ARGS__);                         \
    else if ((k) <= 8) FR_KC_LAUNCH(8, V_, grid, KERNEL, WT, NEG, __VA_ARGS__);                         \
    else if ((k) <= 16) FR_KC_LAUNCH(16, V_, grid, KERNEL, WT, NEG, __VA_ARGS__);                       \
    else if ((k) <= 32) FR_KC_LAUNCH(32, V_, grid, KERNEL, WT, NEG, __VA_ARGS__);                       \
    else FR_KC_LAUNCH(64, V_, grid, KERNEL, WT, NEG, __VA_ARGS__);                                      \
  } while (0)
#define FR_KC_DISPATCH(k, vec, grid, KERNEL, WT, NEG, ...)                                              \
  do {                                                                                                  \
    if (vec) FR_KC_CASES(k, true, grid, KERNEL, WT, NEG, __VA_ARGS__);                                  \
    else FR_KC_CASES(k, false, grid, KERNEL, WT, NEG, __VA_ARGS__);                                     \
  } while (0)

// the FP32-basis kernels KERNEL<KC, NEG> with the smallest KC >= k
#define FR_KC32_LAUNCH(KC_, NEG_, grid, KERNEL, ...) \
  KERNEL<KC_, NEG_><<<wave_grid<KERNEL<KC_, NEG_>>(grid), kRedThreads, 0, s>>>(__VA_ARGS__)
#define FR_KC32_CASES(k, NEG_, grid, KERNEL, ...)                        \
  do {                                                                  \
    if ((k) <= 1) FR_KC32_LAUNCH(1, NEG_, grid, KERNEL, __VA_ARGS__);   \
    else if ((k) <= 2) FR_KC32_LAUNCH(2, NEG_, grid, KERNEL, __VA_ARGS__); \
    else if ((k) <= 4) FR_KC32_LAUNCH(4, NEG_, grid, KERNEL, __VA_ARGS__); \
    else if ((k) <= 8) FR_KC32_LAUNCH(8, NEG_, grid, KERNEL, __VA_ARGS__); \
    else if ((k) <= 16) FR_KC32_LAUNCH(16, NEG_, grid, KERNEL, __VA_ARGS__); \
    else if ((k) <= 32) FR_KC32_LAUNCH(32, NEG_, grid, KERNEL, __VA_ARGS__); \
    else FR_KC32_LAUNCH(64, NEG_, grid, KERNEL, __VA_ARGS__);            \
  } while (0)
#define FR_KC32_DISPATCH(k, neg, grid, KERNEL, ...)               \
  do {                                                           \
    if (neg) FR_KC32_CASES(k, true, grid, KERNEL, __VA_ARGS__);  \
    else FR_KC32_CASES(k, false, grid, KERNEL, __VA_ARGS__);     \
  } while (0)

// smallest GMRES tolerance run with the FP32 Krylov basis
constexpr double kF32BasisMinRtol = 1e-4;

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// column stride of the Krylov basis: n_dof_capacity rounded up to 32 values,
// so that every column starts on a 256-byte boundary
static int64_t krylov_ld(const fr_ctx* c) { return (c->n_dof_cap + 31) & ~(int64_t)31; }

__global__ void k_scale(const double* __restrict__ x, double a, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// x += sum_kk y[kk] V[kk]   (y on the device)
// x (+)= sum_kk y[kk] V[kk]; accumulate 0 (the first cycle) writes x
__global__ void k_combine(const double* __restrict__ V, int64_t ldv, int k, const double* __restrict__ y,
                          double* __restrict__ x, int64_t n, int accumulate) {
  __shared__ double ys[kMaxK];
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = accumulate ? x[i] : 0.0;
    for (int kk = 0; kk < k; ++kk) s += ys[kk] * V[kk * ldv + i];
    x[i] = s;
  }
}

// out = sigma v - J   (J in FP64 or FP32)
template <typename T>
__global__ void k_shift(double sigma, const double* __restrict__ v, const T* __restrict__ J,
                        double* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = sigma * v[i] - (double)J[i];
}

// F = -q / (w dt) + R + rhs (R in FP64 or FP32) and ||F||^2 summed on the
// way (FP64, the deterministic grid reduction into out[0]): the stage
// residual and its norm in one pass
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_stage_F_norm(const double* __restrict__ q, const T* __restrict__ R,
                                                               const double* __restrict__ rhs, double inv_wdt,
                                                               double* __restrict__ F, int64_t n,
                                                               double* __restrict__ partial, double* __restrict__ out,
                                                               unsigned* __restrict__ ticket) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double f = -q[i] * inv_wdt + (double)R[i] + rhs[i];
    F[i] = f;
    acc = fma(f, f, acc);
  }
  const double a1[1] = {acc};
  grid_sum<1>(a1, 1, partial, out, ticket);
}

static unsigned egrid(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
}

// k dot products V[0..k)^T w (or ||w||^2 when V is null) -> host array out[k]
static fr_status multidot(fr_ctx* c, const double* V, int64_t ldv, int k, const double* w, int64_t n,
                          double* out_host, cudaStream_t s) {
  double* part = c->d_red;
  double* dout = c->d_red + kOutH1;
  const int kk = V ? k : 1;
  const bool vec = aligned16(w) && (!V || (aligned16(V) && ldv % 2 == 0));
  const unsigned g = red_blocks(n);
  FR_LAUNCH_B(c, "arnoldi_dot", s, 8.0 * n * ((V ? k : 0) + 1),
              FR_KC_DISPATCH(kk, vec, g, k_multidot, double, false, V, ldv, kk, w, n, part, dout, ticket_of(c), 0,
                             nullptr));
  cudaMemcpyAsync(c->h_red, dout, sizeof(double) * (V ? k : 1), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "multidot");
  std::memcpy(out_host, c->h_red, sizeof(double) * (V ? k : 1));
  return FR_OK;
}

static fr_status norm2(fr_ctx* c, const double* w, int64_t n, double* out, cudaStream_t s) {
  double v;
  fr_status st = multidot(c, nullptr, 0, 1, w, n, &v, s);
  *out = std::sqrt(v);
  return st;
}

// x = (T)(s_j V[j]) with j = *jidx and s_j = scale[j]: the orthonormal Krylov
// vector from its stored column (FP32: the scale applied after the rounding)
template <typename T, typename VT>
__global__ void k_gather_col(const VT* __restrict__ V, int64_t ld, const int* __restrict__ jidx,
                             const double* __restrict__ scale, T* __restrict__ x, int64_t n,
                             const int* __restrict__ gate) {
  if (gate && *gate) return;
  const int j = *jidx;
  const VT* src = V + (int64_t)j * ld;
  const T sc = (T)scale[j];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (T)src[i] * sc;
}

// One Arnoldi product w = -J(q) v_j of the exact mode, v_j = s_j V[j]: gather
// into a fixed buffer (j read from device memory), then the JVP kernels (q
// traces prepared beforehand), whose volume kernel writes -J v_j in FP64
// straight into w.  Replayed from a CUDA graph captured on first use and again
// whenever q, V, w or the timing state changed (the layout and the launch
// tuning drop it); launched directly when graphs are off or cannot be used.
static void gather_col(fr_ctx* c, int pi, const void* V, bool b32, int64_t ld, void* x, int64_t n, cudaStream_t s) {
  const double nb = (double)n * ((b32 ? 4 : 8) + (pi ? 4 : 8));
  const double* sc = c->d_red + kOutS;
  if (b32)
    FR_LAUNCH_B(c, "vec", s, nb,
                k_gather_col<float, float><<<egrid(n), 256, 0, s>>>((const float*)V, ld, c->d_jidx, sc, (float*)x, n,
                                                                   c->gate));
  else if (pi)
    FR_LAUNCH_B(c, "vec", s, nb,
                k_gather_col<float, double><<<egrid(n), 256, 0, s>>>((const double*)V, ld, c->d_jidx, sc, (float*)x,
                                                                    n, c->gate));
  else
    FR_LAUNCH_B(c, "vec", s, nb,
                k_gather_col<double, double><<<egrid(n), 256, 0, s>>>((const double*)V, ld, c->d_jidx, sc,
                                                                     (double*)x, n, c->gate));
}

static void release_graph_timers(fr_ctx* c, int pi) {
  for (auto& r : c->graph_timers[pi]) c->timing.give_back(r);
  c->graph_timers[pi].clear();
}

// The column index is read from c->d_jidx: the caller sets it (the update
// of the previous Arnoldi step stores it on the device).  graph_ok false:
// direct launches (the device-driven cycle, whose launches carry the gate and
// need events of their own for every product).  b32: FP32 basis V, and w
// receives J v in FP32 (the Arnoldi kernels negate it); else FP64 basis and
// w = -J v in FP64.  col >= 0 (direct launches whose basis has the products'
// precision): the product reads the stored column u_col itself, no gather
// runs, and the volume kernel multiplies J u_col by the column's scale s_col
// read on the device (J is linear; the stored columns are unnormalised, so
// the scale has to enter: products of u_col alone would grow the next column
// by |J| every iteration).
static fr_status exact_product(fr_ctx* c, const fr_shifted_op* op, const void* V, void* w, cudaStream_t s,
                               bool graph_ok = true, bool b32 = false, int col = -1) {
  const int pi = op->jv_prec == FR_F64 ? 0 : 1;   // FP32 kernels for FR_F32 and FR_BF16OP
  const fr_prec prec = op->jv_prec;
  const int64_t n = c->n_dof, ld = krylov_ld(c);
  // the q the traces were prepared from: the FP32 copy for FP32 products
  const void* qptr = pi ? (const void*)vec32(c, 0) : (const void*)op->q64_dev;
  void* x = pi ? (void*)vec32(c, 1) : (void*)vec64(c, 10);
  if (!qptr || !x) return FR_ERR_NOMEM;
  collect_graph_timers(c);
  auto direct = [&](cudaStream_t st) -> fr_status {
    gather_col(c, pi, V, b32, ld, x, n, st);
    if (b32) return launch_jvp_prepared(c, qptr, x, w, prec, st);
    return launch_jvp_prepared_neg64(c, qptr, x, (double*)w, prec, st);
  };
  if (col >= 0 && (b32 ? pi == 1 : pi == 0)) {
    const void* vcol = b32 ? (const void*)((const float*)V + (int64_t)col * ld)
                           : (const void*)((const double*)V + (int64_t)col * ld);
    c->vscale = c->d_red + kOutS + col;
    const fr_status e = b32 ? launch_jvp_prepared(c, qptr, vcol, w, prec, s)
                            : launch_jvp_prepared_neg64(c, qptr, vcol, (double*)w, prec, s);
    c->vscale = nullptr;
    return e;
  }
  if (!graph_ok || !c->use_graphs || !c->jvp_graph_ok) return direct(s);
  // the graph holds the event nodes of the kernels timed when it was captured
  const void* timed = c->timing.on ? (const void*)(intptr_t)(1 + c->timing.select_gen) : nullptr;
  const void* key[5] = {qptr, V, w, timed, (const void*)(intptr_t)(prec + 1)};
  if (c->jvp_graph[pi] && std::equal(key, key + 5, c->jvp_graph_key[pi])) {
    if (cudaGraphLaunch(c->jvp_graph[pi], s) != cudaSuccess) {
      cudaGetLastError();
      c->jvp_graph_ok = false;
      return direct(s);
    }
    c->timing.launches += c->jvp_graph_nodes[pi];
    c->graph_timers_live[pi] = c->timing.on && !c->graph_timers[pi].empty();
    return FR_OK;
  }
  if (c->jvp_graph[pi]) {
    cudaStreamSynchronize(s);
    cudaGraphExecDestroy(c->jvp_graph[pi]);
    c->jvp_graph[pi] = nullptr;
    release_graph_timers(c, pi);
  }
  // this product launched directly: every lazy allocation and kernel attribute
  // is then in place before the capture
  fr_status e = direct(s);
  if (e != FR_OK) return e;
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "gmres product");
  // captured on a private stream (the caller's may be the legacy default
  // stream, which cannot be captured); replayed on the caller's stream
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
    c->jvp_graph_ok = false;
    return FR_OK;
  }
  cudaStream_t cs = c->cap_stream;
  const long long l0 = c->timing.launches;
  c->timing.capture = true;
  c->timing.mark = (int64_t)c->timing.pending.size();
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    const fr_status st = direct(cs);
    const cudaError_t ee = cudaStreamEndCapture(cs, &g);
    ok = st == FR_OK && ee == cudaSuccess && g != nullptr && cudaGraphInstantiate(&c->jvp_graph[pi], g, 0) == cudaSuccess;
  }
  if (g) cudaGraphDestroy(g);
  c->timing.capture = false;
  // the timers recorded during the capture belong to the graph
  auto& pend = c->timing.pending;
  c->graph_timers[pi].assign(pend.begin() + c->timing.mark, pend.end());
  pend.resize(c->timing.mark);
  c->jvp_graph_nodes[pi] = (int)(c->timing.launches - l0);
  c->timing.launches = l0;
  if (!ok) {
    cudaGetLastError();
    release_graph_timers(c, pi);
    c->jvp_graph[pi] = nullptr;
    c->jvp_graph_ok = false;
    return FR_OK;   // the direct launches above already produced w
  }
  std::copy(key, key + 5, c->jvp_graph_key[pi]);
  return FR_OK;
}

// y = A x = sigma x - J(q) x, or y = -J(q) x when shifted is false (Arnoldi
// runs on -J: the Krylov space of sigma I - J is that of -J, and the shift is
// added to the Hessenberg diagonal; this avoids the cancellation of w ~ sigma v)
static fr_status apply_op(fr_ctx* c, const fr_shifted_op* op, const double* R0, const double* x, double* y,
                          cudaStream_t s, bool shifted = true) {
  const int64_t n = c->n_dof;
  const double sigma = shifted ? op->sigma : 0.0;
  if (op->mode == FR_JV_FD) {
    double* J = vec64(c, 3);
    if (!J) return FR_ERR_NOMEM;
    fr_status st = launch_fd_jv(c, op->q64_dev, x, J, op->eps, R0, s);
    if (st != FR_OK) return st;
    FR_LAUNCH_B(c, "vec", s, 24.0 * n, k_shift<double><<<egrid(n), 256, 0, s>>>(sigma, x, J, y, n));
  } else if (op->jv_prec == FR_F64) {
    double* J = vec64(c, 3);
    if (!J) return FR_ERR_NOMEM;
    fr_status st = launch_jvp_prepared(c, op->q64_dev, x, J, FR_F64, s);
    if (st != FR_OK) return st;
    FR_LAUNCH_B(c, "vec", s, 24.0 * n, k_shift<double><<<egrid(n), 256, 0, s>>>(sigma, x, J, y, n));
  } else {
    float* q32 = vec32(c, 0);
    float* x32 = vec32(c, 1);
    float* J32 = vec32(c, 2);
    if (!q32 || !x32 || !J32) return FR_ERR_NOMEM;
    vcast_f64_f32(c, x, x32, n, s);
    fr_status st = launch_jvp_prepared(c, q32, x32, J32, op->jv_prec, s);
    if (st != FR_OK) return st;
    FR_LAUNCH_B(c, "vec", s, 20.0 * n, k_shift<float><<<egrid(n), 256, 0, s>>>(sigma, x, J32, y, n));
  }
  return cuda_check(cudaGetLastError(), "shifted operator");
}

// GMRES(m) with x0 = 0.  R0 (optional) = R(q) for the finite-difference mode.
// b_norm: ||b|| when the caller already has it, else negative.
// sync_at_end: return only when x is complete (the public call); the stage
// passes false and lets its next residual overlap the final combination.
// add_to (optional): when the first cycle converges, the combination adds
// V y to *add_to instead of writing x (x is then left as it was) and
// *applied is set; otherwise x is written as usual.
static fr_status gmres_impl(fr_ctx* c, const fr_shifted_op* op, const double* R0, const double* b, double* x,
                            const fr_gmres_opts* o, fr_gmres_stats* st, cudaStream_t s, double b_norm = -1.0,
                            bool sync_at_end = true, double* add_to = nullptr, bool* applied = nullptr) {
  if (applied) *applied = false;
  const int m = o->m;
  const int64_t n = c->n_dof, ld = krylov_ld(c);
  if (m < 1 || m + 1 > kMaxK || o->max_it < 1 || !(o->rtol > 0.0) || o->reorth < 0 || o->reorth > 2) {
    set_error("gmres_solve: need 1 <= m <= 63, max_it >= 1, rtol > 0, reorth in {0, 1, 2}");
    return FR_ERR_INVALID;
  }
  if (op->precond && !c->pc_ready) {
    set_error("gmres_solve: preconditioning requested but no element-Jacobi blocks are built for this layout");
    return FR_ERR_INVALID;
  }
  if (ensure_red(c) != FR_OK) return FR_ERR_NOMEM;
  if (!c->d_jidx) {   // index of the column the next Arnoldi product reads
    if (cudaMalloc(&c->d_jidx, sizeof(int)) != cudaSuccess) return FR_ERR_NOMEM;
    if (cudaMallocHost(&c->h_jidx, sizeof(int) * kMaxK) != cudaSuccess) return FR_ERR_NOMEM;
    for (int k = 0; k < kMaxK; ++k) c->h_jidx[k] = k;
  }
  // FP32 basis: exact FP32 products and a tolerance they can meet (the
  // attainable accuracy of both is about 1e-6); the element-Jacobi
  // preconditioner then works on the FP32 vectors (its sums are FP32 anyway)
  const bool b32 = c->f32_basis && op->mode == FR_JV_EXACT && op->jv_prec != FR_F64 && o->rtol >= kF32BasisMinRtol;
  if (!b32 && (!c->d_krylov || c->krylov_m < m)) {
    cudaFree(c->d_krylov);
    c->d_krylov = nullptr;
    if (cudaMalloc(&c->d_krylov, sizeof(double) * (m + 1) * ld) != cudaSuccess) {
      set_error("gmres_solve: Krylov basis allocation failed");
      return FR_ERR_NOMEM;
    }
    c->krylov_m = m;
    clear_graphs(c);
  }
  if (b32 && (!c->d_krylov32 || c->krylov32_m < m)) {
    cudaFree(c->d_krylov32);
    c->d_krylov32 = nullptr;
    if (cudaMalloc(&c->d_krylov32, sizeof(float) * (m + 1) * ld) != cudaSuccess) {
      set_error("gmres_solve: Krylov basis allocation failed");
      return FR_ERR_NOMEM;
    }
    c->krylov32_m = m;
    clear_graphs(c);
  }
  if (op->mode == FR_JV_EXACT && op->jv_prec != FR_F64) {
    float* q32 = vec32(c, 0);
    if (!q32) return FR_ERR_NOMEM;
    vcast_f64_f32(c, op->q64_dev, q32, n, s);
    fr_status ps = launch_jvp_prepare(c, q32, op->jv_prec, s);
    if (ps != FR_OK) return ps;
  } else if (op->mode == FR_JV_EXACT) {
    fr_status ps = launch_jvp_prepare(c, op->q64_dev, FR_F64, s);
    if (ps != FR_OK) return ps;
  }
  // The Krylov basis is stored unnormalised: column j holds u_j and the
  // orthonormal vector is v_j = s_j u_j, with the scales s_j kept on the host
  // and on the device.  The normalisation pass of every iteration then
  // disappears: the update writes the new column directly, the dots are
  // scaled on the host, the update applies s_i^2 to its coefficients, and the
  // gather in front of the JVP applies s_j.  In the exact modes the JVP's
  // volume kernel writes w = -J v_j in FP64 directly.
  double* V = c->d_krylov;
  float* V32 = c->d_krylov32;
  float* w32 = b32 ? vec32(c, 2) : nullptr;   // J v of the FP32 products (the FP32 basis)
  if (b32 && !w32) return FR_ERR_NOMEM;
  double* w = vec64(c, 4);
  double* r = vec64(c, 5);
  double* xs = vec64(c, 10);   // s_j u_j for the finite-difference product
  double* ydev = c->d_red + kOutY;
  double* sdev = c->d_red + kOutS;
  double* sh = c->h_red + 3 * kMaxK;   // pinned host copy of the scales
  if (!w || !r || !xs) return FR_ERR_NOMEM;
  std::memset(st, 0, sizeof(*st));
  // x0 = 0: the residual of the first cycle is b (left preconditioning: GMRES
  // on M^-1 (sigma I - J) x = M^-1 b, so M^-1 b), read in place; the first
  // combination writes x, later ones add to it
  const bool pc = op->precond != 0;
  double beta0 = pc ? -1.0 : b_norm;
  fr_status e = FR_OK;
  if (pc && (e = precond_apply(c, 1.0, b, 0.0, nullptr, r, s)) != FR_OK) return e;
  const double* r0 = pc ? r : b;
  if (!(beta0 >= 0.0) && (e = norm2(c, r0, n, &beta0, s)) != FR_OK) return e;
  if (!std::isfinite(beta0)) {
    set_error("gmres_solve: non-finite right-hand side");
    return FR_ERR_NONFINITE;
  }
  if (beta0 == 0.0) {
    st->converged = 1;
    cudaMemsetAsync(x, 0, sizeof(double) * n, s);
    return cuda_check(cudaStreamSynchronize(s), "gmres");
  }
  int it = 0;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m), h(kMaxK), h2(kMaxK);
  double res = beta0;
  const bool exact = op->mode == FR_JV_EXACT;
  const bool vec = aligned16(w) && aligned16(V) && ld % 2 == 0;
  const unsigned grid = red_blocks(n);
  unsigned* ticket = ticket_of(c);
  double* part = c->d_red;
  auto set_scale = [&](int j, double v) {
    sh[j] = v;
    cudaMemcpyAsync(sdev + j, sh + j, sizeof(double), cudaMemcpyHostToDevice, s);
  };
  // one Gram-Schmidt pass against columns 0..kk-1: dots of w_in into `raw`,
  // then w_out = w_in - sum s_i^2 raw_i u_i with ||w_out||^2 into N
  // (the update also stores the scale of the new column and the index of
  // the next product on the device: kk is the new column's index)
  auto gs_pass = [&](int kk, const double* w_in, double* w_out, double* raw, int with_norm, StepArgs step) {
    if (c->df_arnoldi)
      FR_LAUNCH_B(c, "arnoldi_dot", s, 8.0 * n * (kk + 1),
                  FR_KC_DISPATCH(kk, vec, grid, k_multidot_df, double, false, V, ld, kk, w_in, n, part, raw, ticket,
                                 with_norm, c->gate));
    else
      FR_LAUNCH_B(c, "arnoldi_dot", s, 8.0 * n * (kk + 1),
                  FR_KC_DISPATCH(kk, vec, grid, k_multidot, double, false, V, ld, kk, w_in, n, part, raw, ticket,
                                 with_norm, c->gate));
    FR_LAUNCH_B(c, "arnoldi_update", s, 8.0 * n * (kk + 2),
                FR_KC_DISPATCH(kk, vec, grid, k_orth_update, double, false, V, ld, kk, raw, sdev, w_in, w_out, n,
                               part, c->d_red + kOutN, ticket, sdev + kk, c->d_jidx, kk, c->gate, step));
  };
  auto gs_pass32 = [&](int kk, const float* w_in, bool neg, float* w_out, double* raw, int with_norm,
                       StepArgs step) {
    FR_LAUNCH_B(c, "arnoldi_dot", s, 4.0 * n * (kk + 1),
                FR_KC32_DISPATCH(kk, neg, grid, k_multidot32, V32, ld, kk, w_in, n, part, raw, ticket, with_norm,
                                 c->gate));
    FR_LAUNCH_B(c, "arnoldi_update", s, 4.0 * n * (kk + 2),
                FR_KC32_DISPATCH(kk, neg, grid, k_orth_update32, V32, ld, kk, raw, sdev, w_in, w_out, n, part,
                                 c->d_red + kOutN, ticket, sdev + kk, c->d_jidx, kk, c->gate, step));
  };
  // the first Gram-Schmidt pass of column kk, on the product's output; a
  // further pass works on the new column in place; `step` (device-driven
  // cycles): the Givens bookkeeping run by the update that ends the iteration
  auto gs_first = [&](int kk, double* raw, int with_norm, StepArgs step = {}) {
    // FP32 basis: w32 holds J v, or M^-1 (sigma v - J v) once preconditioned
    if (b32) gs_pass32(kk, w32, !op->precond, V32 + (int64_t)kk * ld, raw, with_norm, step);
    else gs_pass(kk, w, V + (int64_t)kk * ld, raw, with_norm, step);
  };
  auto gs_again = [&](int kk, double* raw, StepArgs step = {}) {
    if (b32) gs_pass32(kk, V32 + (int64_t)kk * ld, false, V32 + (int64_t)kk * ld, raw, 0, step);
    else gs_pass(kk, V + (int64_t)kk * ld, V + (int64_t)kk * ld, raw, 0, step);
  };
  const void* Vb = b32 ? (const void*)V32 : (const void*)V;
  void* wb = b32 ? (void*)w32 : (void*)w;
  // Device-driven cycle (exact products, one or two Gram-Schmidt passes): the
  // host launches the Arnoldi iterations in batches without waiting between
  // them.  Each iteration is the product, the preconditioner and the
  // Gram-Schmidt pass(es); the block that completes the last update keeps the
  // Hessenberg column, the Givens rotations and the residual estimate on the
  // device (arnoldi_step_block) and closes the gate when the cycle has
  // converged; every later launch of the batch then returns at entry.  The
  // host reads the cycle state once per batch.  A launch past the gate still
  // costs its grid's start-up (about 20 us for a volume kernel of 32,768
  // CTAs against a few us of host round trip), so the first batch is one
  // iteration shorter than the previous cycle and later batches are single
  // iterations.  Timing records of launches past the gate are dropped, so the
  // per-kernel counts hold only iterations that ran.
  const bool dev = c->device_gmres && exact && o->reorth != 1;
  auto drop_timers_from = [&](int64_t mark_p, long long mark_l) {
    auto& pend = c->timing.pending;
    for (int64_t i = mark_p; i < (int64_t)pend.size(); ++i) c->timing.give_back(pend[i]);
    if ((int64_t)pend.size() > mark_p) pend.resize(mark_p);
    c->timing.launches = mark_l;
  };
  auto device_cycle = [&](double beta, int& k, double& res_out) -> fr_status {
    if (!c->d_gm) {
      if (cudaMalloc(&c->d_gm, sizeof(double) * kGmSize) != cudaSuccess) return FR_ERR_NOMEM;
      if (cudaMallocHost(&c->h_gm, sizeof(double) * kGmSize) != cudaSuccess) return FR_ERR_NOMEM;
    }
    double* gm = c->d_gm;
    int* ctl = reinterpret_cast<int*>(gm + kGmCtl);
    const int* hctl = reinterpret_cast<const int*>(c->h_gm + kGmCtl);
    c->h_gm[kGmG] = beta;
    cudaMemcpyAsync(gm + kGmG, c->h_gm + kGmG, sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(ctl, 0, 2 * sizeof(double), s);
    const int jmax = std::min(m, o->max_it - it);
    std::vector<int64_t> mark_p(m + 1, 0);
    std::vector<long long> mark_l(m + 1, 0);
    int batch = std::max(1, std::min(jmax, c->gm_last_k - 1));
    // products straight from the stored columns when the basis has the
    // products' precision (no gather; the volume kernel applies the scale)
    const bool direct_col = b32 ? op->jv_prec != FR_F64 : op->jv_prec == FR_F64;
    int j = 0;
    fr_status ee = FR_OK;
    k = 0;
    while (true) {
      const int jend = std::min(jmax, j + batch);
      c->gate = ctl;
      for (; j < jend && ee == FR_OK; ++j) {
        mark_p[j] = (int64_t)c->timing.pending.size();
        mark_l[j] = c->timing.launches;
        if (j == 0) cudaMemcpyAsync(c->d_jidx, c->h_jidx, sizeof(int), cudaMemcpyHostToDevice, s);
        if ((ee = exact_product(c, op, Vb, wb, s, false, b32, direct_col ? j : -1)) != FR_OK) break;
        if (pc && b32 &&
            (ee = precond_apply(c, -1.0, w32, op->sigma, V32 + (int64_t)j * ld, w32, s, ctl, sdev + j)) != FR_OK)
          break;
        if (pc && !b32 &&
            (ee = precond_apply(c, 1.0, w, op->sigma, V + (int64_t)j * ld, w, s, ctl, sdev + j)) != FR_OK)
          break;
        const int kk = j + 1;
        StepArgs step;
        step.gm = gm;
        step.dots1 = c->d_red + kOutH1;
        step.dots2 = c->d_red + kOutH2;
        step.scale = sdev;
        step.nrm2 = c->d_red + kOutN;
        step.shift = pc ? 0.0 : op->sigma;
        step.tol = o->rtol * beta0;
        step.j = j;
        step.last = it + kk >= o->max_it;
        step.two_pass = o->reorth == 2;
        if (o->reorth == 2) {
          gs_first(kk, c->d_red + kOutH1, 0);
          gs_again(kk, c->d_red + kOutH2, step);
        } else {
          gs_first(kk, c->d_red + kOutH1, 0, step);
        }
      }
      c->gate = nullptr;
      if (ee != FR_OK) return ee;
      mark_p[j] = (int64_t)c->timing.pending.size();
      mark_l[j] = c->timing.launches;
      cudaMemcpyAsync(c->h_gm, gm, sizeof(double) * kGmSize, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(sh, sdev, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "gmres");
      k = hctl[1];
      if (k < j) drop_timers_from(mark_p[k], mark_l[k]);
      if (hctl[2]) {
        set_error("gmres_solve: non-finite Arnoldi vector");
        return FR_ERR_NONFINITE;
      }
      if (hctl[0] || j >= jmax) break;
      batch = 1;
    }
    c->gm_last_k = std::max(1, k);
    // the rotated Hessenberg (row-major, as the host-driven cycle keeps it) and g
    for (int jj = 0; jj < k; ++jj)
      for (int i = 0; i <= jj; ++i) H[i * m + jj] = c->h_gm[kGmH + (int64_t)jj * kMaxK + i];
    for (int i = 0; i <= k; ++i) g[i] = c->h_gm[kGmG + i];
    res_out = std::fabs(g[k]);
    return FR_OK;
  };
  bool first = true;
  while (true) {
    double beta = beta0;   // r = b on the first cycle
    if (!first && (e = norm2(c, r, n, &beta, s)) != FR_OK) return e;
    first = false;
    if (beta <= o->rtol * beta0) {
      st->converged = 1;
      res = beta;
      break;
    }
    if (it >= o->max_it) {
      res = beta;
      break;
    }
    const double* rc = st->restarts == 0 ? r0 : r;
    if (b32) FR_LAUNCH_B(c, "vec", s, 12.0 * n, k_scale32<<<egrid(n), 256, 0, s>>>(rc, 1.0 / beta, V32, n));
    else FR_LAUNCH_B(c, "vec", s, 16.0 * n, k_scale<<<egrid(n), 256, 0, s>>>(rc, 1.0 / beta, V, n));
    set_scale(0, 1.0);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    res = beta;
    if (dev) {
      if ((e = device_cycle(beta, k, res)) != FR_OK) return e;
      it += k;
    }
    for (int j = 0; !dev && j < m; ++j) {
      // product w = -J v_j
      if (exact) {
        if (j == 0) cudaMemcpyAsync(c->d_jidx, c->h_jidx, sizeof(int), cudaMemcpyHostToDevice, s);
        if ((e = exact_product(c, op, Vb, wb, s, true, b32)) != FR_OK) return e;
      } else {
        FR_LAUNCH_B(c, "vec", s, 16.0 * n, k_scale<<<egrid(n), 256, 0, s>>>(V + (int64_t)j * ld, sh[j], xs, n));
        if ((e = apply_op(c, op, R0, xs, w, s, false)) != FR_OK) return e;
      }
      if (pc && b32 && (e = precond_apply(c, -1.0, w32, op->sigma * sh[j], V32 + (int64_t)j * ld, w32, s)) != FR_OK)
        return e;
      if (pc && !b32 && (e = precond_apply(c, 1.0, w, op->sigma * sh[j], V + (int64_t)j * ld, w, s)) != FR_OK)
        return e;
      ++it;
      // classical Gram-Schmidt: one pass (reorth 0), a second pass when the
      // first removed more than half of ||w||^2, ||w_new|| < 0.7 ||w|| (DGKS,
      // reorth 1), or always two passes (reorth 2).  Each pass is one multi-dot
      // and one update, both ending in a grid reduction; the first writes the
      // new column u_{j+1}, the second works on it in place.
      const int kk = j + 1;
      const int ro = o->reorth;
      gs_first(kk, c->d_red + kOutH1, ro == 1 ? 1 : 0);
      if (ro == 2) gs_again(kk, c->d_red + kOutH2);
      cudaMemcpyAsync(c->h_red, c->d_red + kOutH1, sizeof(double) * 3 * kMaxK, cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "gmres");
      for (int i = 0; i <= j; ++i) {
        h[i] = sh[i] * c->h_red[i];
        h2[i] = ro == 2 ? sh[i] * c->h_red[kMaxK + i] : 0.0;
      }
      if (ro == 1 && std::sqrt(c->h_red[2 * kMaxK]) < 0.7 * std::sqrt(c->h_red[kk])) {
        gs_again(kk, c->d_red + kOutH2);
        cudaMemcpyAsync(c->h_red + kMaxK, c->d_red + kOutH2, sizeof(double) * 2 * kMaxK, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "gmres");
        for (int i = 0; i <= j; ++i) h2[i] = sh[i] * c->h_red[kMaxK + i];
      }
      const double hn = std::sqrt(c->h_red[2 * kMaxK]);
      for (int i = 0; i <= j; ++i) H[i * m + j] = h[i] + h2[i];
      if (!pc) H[j * m + j] += op->sigma;   // Hessenberg of sigma I - J from that of -J
      H[(j + 1) * m + j] = hn;
      if (!std::isfinite(hn)) {
        set_error("gmres_solve: non-finite Arnoldi vector");
        return FR_ERR_NONFINITE;
      }
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      if (den == 0.0) {
        cs[j] = 1.0;
        sn[j] = 0.0;
      } else {
        cs[j] = H[j * m + j] / den;
        sn[j] = H[(j + 1) * m + j] / den;
      }
      H[j * m + j] = cs[j] * H[j * m + j] + sn[j] * H[(j + 1) * m + j];
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      res = std::fabs(g[j + 1]);
      k = j + 1;
      if (hn != 0.0) sh[j + 1] = 1.0 / hn;   // the device copy was stored by the update
      if (res <= o->rtol * beta0 || it >= o->max_it || hn == 0.0) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < k; ++l) t -= H[i * m + l] * y[l];
      y[i] = t / H[i * m + i];
    }
    // x += sum_i y_i v_i = sum_i (y_i s_i) u_i
    for (int i = 0; i < k; ++i) y[i] *= sh[i];
    cudaMemcpyAsync(ydev, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s);
    // the first cycle converged and the caller wants the correction added to
    // its vector: one pass, x untouched
    const bool direct = add_to && st->restarts == 0 && res <= o->rtol * beta0;
    double* dst = direct ? add_to : x;
    const int acc = direct || st->restarts > 0;
    if (b32)
      FR_LAUNCH_B(c, "arnoldi_update", s, 4.0 * n * k + (acc ? 16.0 : 8.0) * n,
                  k_combine32<<<egrid(n), 256, 0, s>>>(V32, ld, k, ydev, dst, n, acc));
    else
      FR_LAUNCH_B(c, "arnoldi_update", s, 8.0 * n * (k + (acc ? 2 : 1)),
                  k_combine<<<egrid(n), 256, 0, s>>>(V, ld, k, ydev, dst, n, acc));
    if (direct) *applied = true;
    st->restarts += 1;
    if (res <= o->rtol * beta0) {
      st->converged = 1;
      break;
    }
    if (it >= o->max_it) break;
    // true residual at restart (not counted as an iteration)
    if ((e = apply_op(c, op, R0, x, w, s)) != FR_OK) return e;
    cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    vaxpby(c, -1.0, w, 1.0, r, n, s);
    if (pc && (e = precond_apply(c, 1.0, r, 0.0, nullptr, r, s)) != FR_OK) return e;
  }
  st->iterations = it;
  st->rel_res = res / beta0;
  if (!sync_at_end) return cuda_check(cudaGetLastError(), "gmres");
  return cuda_check(cudaStreamSynchronize(s), "gmres");
}

}  // namespace frgb

using namespace frgb;

extern "C" {

fr_status gmres_solve(fr_ctx* c, const fr_shifted_op* op, const double* b_dev, double* x_dev,
                      const fr_gmres_opts* opts, fr_gmres_stats* stats, void* stream) {
  if (!c || !op || !op->q64_dev || !b_dev || !x_dev || !opts || !stats) {
    set_error("gmres_solve: null argument");
    return FR_ERR_INVALID;
  }
  if (op->mode == FR_JV_FD && !(op->eps > 0.0)) {
    set_error("gmres_solve: finite-difference mode needs eps > 0");
    return FR_ERR_INVALID;
  }
  if (op->mode != FR_JV_FD && op->mode != FR_JV_EXACT) {
    set_error("gmres_solve: unknown product mode");
    return FR_ERR_INVALID;
  }
  if (op->jv_prec != FR_F64 && op->jv_prec != FR_F32 && op->jv_prec != FR_BF16OP) {
    set_error("gmres_solve: unknown product precision");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const double* R0 = nullptr;
  if (op->mode == FR_JV_FD) {
    double* r0 = vec64(c, 2);
    if (!r0) return FR_ERR_NOMEM;
    fr_status st = launch_residual(c, op->q64_dev, r0, FR_F64, s);
    if (st != FR_OK) return st;
    R0 = r0;
  }
  return gmres_impl(c, op, R0, b_dev, x_dev, opts, stats, s);
}

fr_status esdirk_stage(fr_ctx* c, const fr_tableau* tab, int32_t stage, double dt, const double* qn_dev,
                       double* const* Rstages_dev, double* qi_dev, const fr_newton_opts* o,
                       fr_stage_stats* st, void* stream) {
  if (!c || !tab || !qn_dev || !qi_dev || !o || !st || tab->s < 2 || tab->s > 6 || stage < 2 ||
      stage > tab->s || !(dt > 0.0) || !(o->tol > 0.0) || !(o->dtau_init > 0.0) || !(o->dtau_max > 0.0) ||
      !(o->low_above >= 0.0) || (o->low_above > 0.0 && o->low_prec != FR_F32 && o->low_prec != FR_DF) ||
      (o->mode != FR_JV_FD && o->mode != FR_JV_EXACT) ||
      (o->jv_prec != FR_F64 && o->jv_prec != FR_F32 && o->jv_prec != FR_BF16OP)) {
    set_error("esdirk_stage: bad argument");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int i = stage - 1;
  const int S = tab->s;
  const double w = tab->A[i * S + i];
  if (!(w > 0.0)) {
    set_error("esdirk_stage: diagonal coefficient must be positive");
    return FR_ERR_INVALID;
  }
  for (int j = 0; j < i; ++j)
    if (tab->A[i * S + j] != 0.0 && (!Rstages_dev || !Rstages_dev[j])) {
      set_error("esdirk_stage: missing R(q^j)");
      return FR_ERR_INVALID;
    }
  const int64_t n = c->n_dof;
  const double inv_wdt = 1.0 / (w * dt);
  double* rhs = vec64(c, 6);
  double* R = vec64(c, 7);
  double* F = vec64(c, 8);
  double* dq = vec64(c, 9);
  if (!rhs || !R || !F || !dq) return FR_ERR_NOMEM;
  fr_status e = ensure_red(c);
  if (e != FR_OK) return e;
  // rhs = (q^n + dt sum_{j<i} a_ij R(q^j)) / (w dt)
  FR_LAUNCH_B(c, "vec", s, 16.0 * n, k_scale<<<egrid(n), 256, 0, s>>>(qn_dev, inv_wdt, rhs, n));
  for (int j = 0; j < i; ++j)
    if (tab->A[i * S + j] != 0.0) vaxpby(c, dt * tab->A[i * S + j] * inv_wdt, Rstages_dev[j], 1.0, rhs, n, s);
  std::memset(st, 0, sizeof(*st));
  // F from the FP64 residual, or (mixed mode, while ||F|| is large) from the
  // double-float residual of the FP64 state or the FP32 residual of the
  // FP32-rounded state; the FP32 buffers are the GMRES product scratch, idle
  // between solves
  const bool mixedF = o->mode == FR_JV_EXACT && o->low_above > 0.0;
  const bool low32 = mixedF && o->low_prec == FR_F32;
  float* q32 = low32 ? vec32(c, 1) : nullptr;
  float* R32 = low32 ? vec32(c, 2) : nullptr;
  if (low32 && (!q32 || !R32)) return FR_ERR_NOMEM;
  bool low = mixedF;
  const unsigned rgrid = red_blocks(n);
  double* nout = c->d_red + kOutH1;
  auto evalF = [&](double* norm) -> fr_status {
    fr_status ee;
    if (low && low32) {
      vcast_f64_f32(c, qi_dev, q32, n, s);
      if ((ee = launch_residual(c, q32, R32, FR_F32, s)) != FR_OK) return ee;
      FR_LAUNCH_B(c, "vec", s, 28.0 * n,
                  k_stage_F_norm<float><<<rgrid, kRedThreads, 0, s>>>(qi_dev, R32, rhs, inv_wdt, F, n, c->d_red, nout,
                                                                       ticket_of(c)));
      st->low_evaluations += 1;
    } else {
      if ((ee = launch_residual(c, qi_dev, R, low ? FR_DF : FR_F64, s)) != FR_OK) return ee;
      FR_LAUNCH_B(c, "vec", s, 32.0 * n,
                  k_stage_F_norm<double><<<rgrid, kRedThreads, 0, s>>>(qi_dev, R, rhs, inv_wdt, F, n, c->d_red, nout,
                                                                        ticket_of(c)));
      if (low) st->low_evaluations += 1;
      else st->f64_evaluations += 1;
    }
    cudaMemcpyAsync(c->h_red, nout, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "stage residual");
    *norm = std::sqrt(c->h_red[0]);
    if (!std::isfinite(*norm)) {
      set_error("esdirk_stage: non-finite stage residual");
      return FR_ERR_NONFINITE;
    }
    return FR_OK;
  };
  double norm;
  if ((e = evalF(&norm)) != FR_OK) return e;
  st->norm0 = norm;
  double dtau = o->dtau_init, norm_prev = -1.0;
  fr_shifted_op op;
  op.q64_dev = qi_dev;
  op.mode = o->mode;
  op.jv_prec = o->mode == FR_JV_FD ? FR_F64 : o->jv_prec;
  op.eps = o->eps;
  op.precond = o->precond;
  for (int m = 0; m < o->max_newton; ++m) {
    // FP64 from here on, starting with this F, once ||F|| is below the
    // threshold, or once an iteration reduced it by less than 10 %: the noise
    // floor of the low-precision residual may lie above the threshold
    if (low && (norm <= o->low_above * st->norm0 || (norm_prev > 0.0 && norm > 0.9 * norm_prev))) {
      low = false;
      if ((e = evalF(&norm)) != FR_OK) return e;
    }
    if (!low && norm <= o->tol * st->norm0) {
      st->converged = 1;
      break;
    }
    if (norm_prev > 0.0) dtau = std::min(dtau * norm_prev / norm, o->dtau_max);
    fr_gmres_stats gs;
    bool applied = false;   // the solve added its correction to q itself
    for (int h = 0; h <= o->max_halvings; ++h) {
      op.sigma = inv_wdt + 1.0 / dtau;
      if ((e = gmres_impl(c, &op, R, F, dq, &o->gmres, &gs, s, norm, false, qi_dev, &applied)) != FR_OK) return e;
      st->gmres_iterations += gs.iterations;
      if (gs.converged) break;
      dtau *= 0.5;
      st->halvings += 1;
    }
    if (!applied) vaxpby(c, 1.0, dq, 1.0, qi_dev, n, s);
    norm_prev = norm;
    if ((e = evalF(&norm)) != FR_OK) return e;
    st->newton_iterations += 1;
  }
  if (low) {   // iteration limit reached in the low-precision phase: the stage ends on an FP64 F
    low = false;
    if ((e = evalF(&norm)) != FR_OK) return e;
  }
  if (norm <= o->tol * st->norm0) st->converged = 1;
  st->norm_final = norm;
  if (Rstages_dev && Rstages_dev[i])
    cudaMemcpyAsync(Rstages_dev[i], R, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  e = cuda_check(cudaStreamSynchronize(s), "esdirk_stage");
  if (e != FR_OK) return e;
  return st->converged ? FR_OK : FR_ERR_NOT_CONVERGED;
}

fr_status esdirk_step(fr_ctx* c, const fr_tableau* tab, double dt, double* q, const fr_newton_opts* o,
                      fr_stage_stats* stats, const fr_adapt_opts* adapt, int32_t adapt_var, void* stream) {
  if (!c || !tab || !q || !o || tab->s < 2 || tab->s > 6 || !(dt > 0.0) ||
      (adapt && (adapt_var < 0 || adapt_var >= c->nv))) {
    set_error("esdirk_step: bad argument");
    return FR_ERR_INVALID;
  }
  const int S = tab->s;
  for (int j = 0; j < S; ++j)
    if (tab->A[j] != 0.0) {
      set_error("esdirk_step: the first stage must be explicit (first row of A zero)");
      return FR_ERR_INVALID;
    }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = c->n_dof, cap = c->n_dof_cap;
  // S stage residuals, q^n, the stage value, and eta (n_elem + 1)
  const int64_t need = (S + 2) * cap + c->E + 1;
  if (c->step_cap < need) {
    cudaFree(c->d_step);
    c->d_step = nullptr;
    c->step_cap = 0;
    if (cudaMalloc(&c->d_step, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      set_error("esdirk_step: workspace allocation failed");
      return FR_ERR_NOMEM;
    }
    c->step_cap = need;
  }
  double* Rst[6] = {};
  for (int i = 0; i < S; ++i) Rst[i] = c->d_step + i * cap;
  double* qn = c->d_step + S * cap;
  double* qi = qn + cap;
  double* eta = qi + cap;
  cudaMemcpyAsync(qn, q, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  fr_status e;
  if (o->precond) {
    // once per physical time step, at q^n, with the largest shift the stages use (Sec. 2.3)
    const double sigma_pc = 1.0 / (tab->A[1 * S + 1] * dt) + 1.0 / o->dtau_max;
    if ((e = fr_precond_build(c, qn, sigma_pc, stream)) != FR_OK) return e;
  }
  e = launch_residual(c, qn, Rst[0], FR_F64, s);
  if (e != FR_OK) return e;
  cudaMemcpyAsync(qi, qn, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  // stage i starts from the value of stage i-1
  for (int i = 2; i <= S; ++i) {
    fr_stage_stats st;
    std::memset(&st, 0, sizeof(st));
    e = esdirk_stage(c, tab, i, dt, qn, Rst, qi, o, &st, stream);
    if (stats) stats[i - 2] = st;
    if (e != FR_OK) return e;
  }
  // q^{n+1} = q^n + dt sum_i b_i R(q^i)
  cudaMemcpyAsync(q, qn, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  for (int i = 0; i < S; ++i)
    if (tab->b[i] != 0.0) vaxpby(c, dt * tab->b[i], Rst[i], 1.0, q, n, s);
  if (adapt) {
    if ((e = spectral_decay_indicator(c, q, FR_F64, adapt_var, eta, eta + c->E, stream)) != FR_OK) return e;
    if ((e = p_rebucket(c, eta, eta + c->E, adapt, q, FR_F64, nullptr, stream)) != FR_OK) return e;
  }
  return cuda_check(cudaStreamSynchronize(s), "esdirk_step");
}

}  // extern "C"
