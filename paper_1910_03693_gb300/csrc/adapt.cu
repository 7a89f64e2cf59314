// p-adaptation (Sec. 3.1) on the device: the spectral decay smoothness
// indicator, the degree decision, the neighbour jump limit, and the
// reordering of elements into (p, element id) buckets with prolongation /
// projection of their state.  This replaces the paper's ParMETIS
// repartition and all-gather redistribution (Sec. 3.2) on one GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fr_launch.h"

namespace frgb {

fr_status build_layout(fr_ctx* c);

// ---------------------------------------------------------------------------
// indicator: eta = sum w|J| (s - s_{p-1})^2 / sum w|J| s^2 with s_{p-1} the
// Legendre truncation that drops every mode with an index equal to p.  One
// thread per element, fixed summation order (deterministic).
// ---------------------------------------------------------------------------
template <typename T, int ND, int P>
__global__ void k_indicator(const T* __restrict__ q, int var, const int32_t* __restrict__ slot_elem,
                            const BasisTab<double>* __restrict__ basis, GeoView<double> geo,
                            int64_t state_base, int count, int slot_begin, double* __restrict__ eta) {
  constexpr int NV = ND + 2;
  constexpr int NSP = ND == 2 ? P * P : P * P * P;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const BasisTab<double>& B = basis[P];
  const int e = slot_elem[slot_begin + i];
  const T* s = q + state_base + ((int64_t)i * NV + var) * NSP;
  double c[NSP], t[NSP];
  for (int k = 0; k < NSP; ++k) c[k] = (double)s[k];
  // modal coefficients, one direction at a time (xi, eta, zeta)
  for (int d = 0; d < ND; ++d) {
    const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
    for (int k = 0; k < NSP; ++k) {
      const int id = (k / stride) % P, base = k - id * stride;
      double acc = 0.0;
      for (int m = 0; m < P; ++m) acc += B.modal[id][m] * c[base + m * stride];
      t[k] = acc;
    }
    for (int k = 0; k < NSP; ++k) c[k] = t[k];
  }
  // keep only the modes with some index equal to p (they are s - s_{p-1})
  for (int k = 0; k < NSP; ++k) {
    const int i0 = k % P, i1 = (k / P) % P, i2 = ND == 3 ? k / (P * P) : 0;
    const bool top = i0 == P - 1 || i1 == P - 1 || (ND == 3 && i2 == P - 1);
    if (!top) c[k] = 0.0;
  }
  for (int d = 0; d < ND; ++d) {
    const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
    for (int k = 0; k < NSP; ++k) {
      const int id = (k / stride) % P, base = k - id * stride;
      double acc = 0.0;
      for (int m = 0; m < P; ++m) acc += B.nodal[id][m] * c[base + m * stride];
      t[k] = acc;
    }
    for (int k = 0; k < NSP; ++k) c[k] = t[k];
  }
  double num = 0.0, den = 0.0;
  for (int k = 0; k < NSP; ++k) {
    const int i0 = k % P, i1 = (k / P) % P, i2 = ND == 3 ? k / (P * P) : 0;
    double w = B.w[i0] * B.w[i1];
    if (ND == 3) w *= B.w[i2];
    w *= geo.vol[(int64_t)e * geo.ves + (int64_t)(ND * ND) * geo.vks + (int64_t)k * geo.vps];
    const double sv = (double)s[k];
    num += w * c[k] * c[k];
    den += w * sv * sv;
  }
  eta[e] = den > 0.0 ? num / den : 0.0;
}

__global__ void k_max_partial(const double* __restrict__ x, int n, double* __restrict__ part) {
  __shared__ double sm[256];
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmax(m, x[i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_max_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double m = 0.0;
    for (int b = 0; b < nb; ++b) m = fmax(m, part[b]);
    out[0] = m;
  }
}

template <typename T, int ND>
static void launch_indicator(fr_ctx* c, const T* q, int var, double* eta, cudaStream_t s) {
  for (const auto& b : c->buckets) {
    GeoView<double> g{};
    const int P = b.p + 1, NKV = geo_nk_vol(c->nd), NKF = geo_nk_face(c->nd);
    int NSP = 1;
    for (int d = 0; d < ND; ++d) NSP *= P;
    if (c->affine) {
      g.vol = c->d_gaff64; g.ves = NKF; g.vks = 1; g.vps = 0;
    } else {
      g.vol = c->d_gvol64[b.p]; g.ves = (int64_t)NKV * NSP; g.vks = NSP; g.vps = 1;
    }
    const unsigned grid = (unsigned)((b.count + 127) / 128);
    const double nb = (double)b.count * NSP * sizeof(T);
#define IND_CASE(PP) \
  case PP: FR_LAUNCH_B(c, "indicator", s, nb, k_indicator<T, ND, PP><<<grid, 128, 0, s>>>(q, var, c->d_slot_elem, c->d_basis64, g, b.state_base, b.count, b.slot_begin, eta)); break;
    switch (P) {
      IND_CASE(2)
      IND_CASE(3)
      IND_CASE(4)
      IND_CASE(5)
      IND_CASE(6)
    }
#undef IND_CASE
  }
}

// Nodal polynomial filter: q <- q - alpha (q - P_{p-1} q) = (1 - alpha) q +
// alpha P_{p-1} q, one thread per (element, variable): modal coefficients
// direction by direction, the modes with some index equal to p kept (they are
// q - P_{p-1} q), back to nodal values, subtracted with weight alpha.
template <int ND, int P>
__global__ void k_filter(double* __restrict__ q, const BasisTab<double>* __restrict__ basis, int64_t state_base,
                         int count, double alpha) {
  constexpr int NV = ND + 2;
  constexpr int NSP = ND == 2 ? P * P : P * P * P;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)count * NV) return;
  const BasisTab<double>& B = basis[P];
  double* s = q + state_base + tid * NSP;   // element tid / NV, variable tid % NV
  double c[NSP], t[NSP];
  for (int k = 0; k < NSP; ++k) c[k] = s[k];
  for (int d = 0; d < ND; ++d) {
    const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
    for (int k = 0; k < NSP; ++k) {
      const int id = (k / stride) % P, base = k - id * stride;
      double acc = 0.0;
      for (int m = 0; m < P; ++m) acc += B.modal[id][m] * c[base + m * stride];
      t[k] = acc;
    }
    for (int k = 0; k < NSP; ++k) c[k] = t[k];
  }
  for (int k = 0; k < NSP; ++k) {
    const int i0 = k % P, i1 = (k / P) % P, i2 = ND == 3 ? k / (P * P) : 0;
    const bool top = i0 == P - 1 || i1 == P - 1 || (ND == 3 && i2 == P - 1);
    if (!top) c[k] = 0.0;
  }
  for (int d = 0; d < ND; ++d) {
    const int stride = d == 0 ? 1 : (d == 1 ? P : P * P);
    for (int k = 0; k < NSP; ++k) {
      const int id = (k / stride) % P, base = k - id * stride;
      double acc = 0.0;
      for (int m = 0; m < P; ++m) acc += B.nodal[id][m] * c[base + m * stride];
      t[k] = acc;
    }
    for (int k = 0; k < NSP; ++k) c[k] = t[k];
  }
  for (int k = 0; k < NSP; ++k) s[k] -= alpha * c[k];
}

// ---------------------------------------------------------------------------
// adaptation
// ---------------------------------------------------------------------------
__global__ void k_decide(const double* __restrict__ eta, const double* __restrict__ eta_max,
                         const int8_t* __restrict__ p_old, double nu_max, double nu_min, int p_min,
                         int p_max, int E, int8_t* __restrict__ p_new) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int p = p_old[e];
  const double em = eta_max[0];
  if (em > 0.0) {
    if (eta[e] > nu_max * em) p += 1;
    if (eta[e] < nu_min * em) p -= 1;
  }
  p = p < p_min ? p_min : (p > p_max ? p_max : p);
  p_new[e] = (int8_t)p;
}

// one Jacobi sweep of p_e <- max(p_e, max_n p_n - 1); *changed set when anything rose
__global__ void k_smooth(const int8_t* __restrict__ p_in, const int32_t* __restrict__ nbr, int nf, int E,
                         int8_t* __restrict__ p_out, int* __restrict__ changed) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int p = p_in[e];
  for (int f = 0; f < nf; ++f) {
    const int n = nbr[(int64_t)e * nf + f];
    if (n >= 0) p = max(p, (int)p_in[n] - 1);
  }
  if (p != p_in[e]) atomicOr(changed, 1);
  p_out[e] = (int8_t)p;
}

// stable counting sort by (p, id): per-block counts of each degree
constexpr int kSortBlock = 1024;
__global__ void k_sort_count(const int8_t* __restrict__ p, int E, int* __restrict__ blk_counts) {
  __shared__ int cnt[kMaxDeg + 1];
  if (threadIdx.x <= kMaxDeg) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int e = blockIdx.x * kSortBlock + threadIdx.x;
  if (e < E) atomicAdd(&cnt[p[e]], 1);
  __syncthreads();
  if (threadIdx.x <= kMaxDeg) blk_counts[blockIdx.x * (kMaxDeg + 1) + threadIdx.x] = cnt[threadIdx.x];
}

// exclusive offsets: blk_off[b][p] = bucket_base[p] + sum_{b' < b} counts[b'][p]
__global__ void k_sort_scan(const int* __restrict__ blk_counts, int nb, int* __restrict__ blk_off,
                            int* __restrict__ totals) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int tot[kMaxDeg + 1] = {0};
  for (int b = 0; b < nb; ++b)
    for (int p = 0; p <= kMaxDeg; ++p) tot[p] += blk_counts[b * (kMaxDeg + 1) + p];
  int base[kMaxDeg + 1];
  int run = 0;
  for (int p = 0; p <= kMaxDeg; ++p) {
    base[p] = run;
    run += tot[p];
    totals[p] = tot[p];
  }
  for (int b = 0; b < nb; ++b)
    for (int p = 0; p <= kMaxDeg; ++p) {
      blk_off[b * (kMaxDeg + 1) + p] = base[p];
      base[p] += blk_counts[b * (kMaxDeg + 1) + p];
    }
}

// rank of each element among the block's elements of its degree (stable)
__global__ void k_sort_scatter(const int8_t* __restrict__ p, int E, const int* __restrict__ blk_off,
                               int32_t* __restrict__ new_slot_elem, int32_t* __restrict__ new_elem_slot) {
  __shared__ int warp_cnt[kSortBlock / 32][kMaxDeg + 1];
  const int e = blockIdx.x * kSortBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pe = e < E ? p[e] : -1;
  int rank_in_warp = 0;
  for (int pp = 0; pp <= kMaxDeg; ++pp) {
    const unsigned m = __ballot_sync(0xffffffffu, pe == pp);
    if (pe == pp) rank_in_warp = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_cnt[warp][pp] = __popc(m);
  }
  __syncthreads();
  if (e >= E) return;
  int before = 0;
  for (int w = 0; w < warp; ++w) before += warp_cnt[w][pe];
  const int slot = blk_off[blockIdx.x * (kMaxDeg + 1) + pe] + before + rank_in_warp;
  new_slot_elem[slot] = e;
  new_elem_slot[e] = slot;
}

// state transfer: one block per new slot; 1D operator applied in each direction
template <typename T, int ND>
__global__ void k_transfer(const T* __restrict__ q_old, T* __restrict__ q_new,
                           const int32_t* __restrict__ new_slot_elem, const int32_t* __restrict__ old_elem_slot,
                           const int64_t* __restrict__ old_state_off, const int8_t* __restrict__ old_slot_p,
                           const int8_t* __restrict__ p_new, const int64_t* __restrict__ new_state_off,
                           const double* __restrict__ xfer, int E) {
  constexpr int NV = ND + 2;
  constexpr int MAXSP = ND == 2 ? 36 : 216;
  __shared__ double a[MAXSP], b[MAXSP];
  const int slot = blockIdx.x;
  if (slot >= E) return;
  const int e = new_slot_elem[slot];
  const int so = old_elem_slot[e];
  const int Po = old_slot_p[so] + 1, Pn = p_new[e] + 1;
  const T* src = q_old + old_state_off[so];
  T* dst = q_new + new_state_off[slot];
  const double* M = xfer + ((size_t)Po * (kPM + 1) + Pn) * kPM * kPM;   // M[i_new][k_old]
  const int nso = ND == 2 ? Po * Po : Po * Po * Po;
  const int nsn = ND == 2 ? Pn * Pn : Pn * Pn * Pn;
  for (int v = 0; v < NV; ++v) {
    for (int k = threadIdx.x; k < nso; k += blockDim.x) a[k] = (double)src[v * nso + k];
    __syncthreads();
    // apply along xi, eta, zeta; sizes change from Po to Pn one axis at a time
    int dims[3] = {Po, Po, ND == 3 ? Po : 1};
    double* in = a;
    double* out = b;
    for (int d = 0; d < ND; ++d) {
      int nd_[3] = {dims[0], dims[1], dims[2]};
      nd_[d] = Pn;
      const int nout = nd_[0] * nd_[1] * nd_[2];
      for (int k = threadIdx.x; k < nout; k += blockDim.x) {
        int i[3] = {k % nd_[0], (k / nd_[0]) % nd_[1], k / (nd_[0] * nd_[1])};
        double acc = 0.0;
        for (int m = 0; m < dims[d]; ++m) {
          int j[3] = {i[0], i[1], i[2]};
          j[d] = m;
          acc += M[i[d] * kPM + m] * in[j[0] + dims[0] * (j[1] + dims[1] * j[2])];
        }
        out[k] = acc;
      }
      __syncthreads();
      dims[d] = Pn;
      double* tmp = in;
      in = out;
      out = tmp;
    }
    for (int k = threadIdx.x; k < nsn; k += blockDim.x) dst[v * nsn + k] = (T)in[k];
    __syncthreads();
  }
}

__global__ void k_new_offsets(const int32_t* __restrict__ new_slot_elem, const int8_t* __restrict__ p_new,
                              const int* __restrict__ totals, int E, int nd, int nv,
                              int64_t* __restrict__ new_state_off) {
  // bucket bases in values, then offset within the bucket
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= E) return;
  const int p = p_new[new_slot_elem[slot]];
  int64_t base = 0;
  int first = 0;
  for (int pp = 0; pp < p; ++pp) {
    const int P = pp + 1;
    const int64_t nsp = nd == 2 ? P * P : P * P * P;
    base += (int64_t)totals[pp] * nv * nsp;
    first += totals[pp];
  }
  const int P = p + 1;
  const int64_t nsp = nd == 2 ? P * P : P * P * P;
  new_state_off[slot] = base + (int64_t)(slot - first) * nv * nsp;
}

static fr_status ensure_transfer_tables(fr_ctx* c, double** out) {
  static_assert(kPM == 6, "transfer table layout");
  if (c->d_xfer) {
    *out = c->d_xfer;
    return FR_OK;
  }
  std::vector<double> h((size_t)(kPM + 1) * (kPM + 1) * kPM * kPM, 0.0);
  for (int Po = 2; Po <= kPM; ++Po)
    for (int Pn = 2; Pn <= kPM; ++Pn) {
      double* M = h.data() + ((size_t)Po * (kPM + 1) + Pn) * kPM * kPM;
      double xo[kPM], wo[kPM], xn[kPM], wn[kPM];
      gauss_legendre(Po, xo, wo);
      gauss_legendre(Pn, xn, wn);
      if (Pn >= Po) {
        // prolongation: interpolate the degree Po-1 polynomial at the new points
        for (int i = 0; i < Pn; ++i) lagrange_eval(xo, Po, xn[i], M + i * kPM);
      } else {
        // projection: Legendre coefficients of the old field, modes < Pn kept
        for (int i = 0; i < Pn; ++i)
          for (int k = 0; k < Po; ++k) {
            double acc = 0.0;
            for (int m = 0; m < Pn; ++m) acc += legendre_p(m, xn[i]) * 0.5 * (2 * m + 1) * wo[k] * legendre_p(m, xo[k]);
            M[i * kPM + k] = acc;
          }
      }
    }
  if (cudaMalloc(&c->d_xfer, sizeof(double) * h.size()) != cudaSuccess) return FR_ERR_NOMEM;
  cudaMemcpy(c->d_xfer, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
  *out = c->d_xfer;
  return FR_OK;
}

}  // namespace frgb

using namespace frgb;

extern "C" {

fr_status spectral_decay_indicator(fr_ctx* c, const void* q_dev, fr_prec prec, int32_t var, double* eta_dev,
                                   double* eta_max_dev, void* stream) {
  if (!c || !q_dev || !eta_dev || (prec != FR_F64 && prec != FR_F32 && prec != FR_BF16OP) || var < 0 || var >= c->nv) {
    set_error("spectral_decay_indicator: bad argument");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (c->nd == 2) {
    if (prec == FR_F64) launch_indicator<double, 2>(c, (const double*)q_dev, var, eta_dev, s);
    else launch_indicator<float, 2>(c, (const float*)q_dev, var, eta_dev, s);
  } else {
    if (prec == FR_F64) launch_indicator<double, 3>(c, (const double*)q_dev, var, eta_dev, s);
    else launch_indicator<float, 3>(c, (const float*)q_dev, var, eta_dev, s);
  }
  if (eta_max_dev) {
    if (!c->d_adapt_f64 && cudaMalloc(&c->d_adapt_f64, sizeof(double) * 1024) != cudaSuccess) return FR_ERR_NOMEM;
    double* part = c->d_adapt_f64;
    FR_LAUNCH(c, "indicator", s, k_max_partial<<<256, 256, 0, s>>>(eta_dev, c->E, part));
    FR_LAUNCH(c, "indicator", s, k_max_final<<<1, 32, 0, s>>>(part, 256, eta_max_dev));
  }
  return cuda_check(cudaGetLastError(), "spectral_decay_indicator");
}

fr_status p_rebucket(fr_ctx* c, const double* eta_dev, const double* eta_max_dev, const fr_adapt_opts* o,
                     void* q_dev, fr_prec prec, int32_t* perm_out_dev, void* stream) {
  if (!c || !eta_dev || !eta_max_dev || !o || !q_dev || (prec != FR_F64 && prec != FR_F32 && prec != FR_BF16OP) ||
      o->p_min < c->p_min || o->p_max > c->p_max || o->p_min > o->p_max) {
    set_error("p_rebucket: bad argument (degrees must lie within the context's limits)");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int E = c->E, nf = c->nf;
  const int nb = (E + kSortBlock - 1) / kSortBlock;
  // integer workspace: p_old, p_a, p_b (bytes) ; counts, offsets, totals, slots (ints)
  if (!c->d_adapt_i32) {
    const size_t ints = (size_t)2 * nb * (kMaxDeg + 1) + (kMaxDeg + 1) + 2 * (size_t)E + 4;
    if (cudaMalloc(&c->d_adapt_i32, sizeof(int) * ints) != cudaSuccess) return FR_ERR_NOMEM;
    if (cudaMalloc(&c->d_adapt_i8, 3 * (size_t)E) != cudaSuccess) return FR_ERR_NOMEM;
    if (!c->d_adapt_f64 && cudaMalloc(&c->d_adapt_f64, sizeof(double) * 1024) != cudaSuccess) return FR_ERR_NOMEM;
    if (cudaMalloc(&c->d_old_state_off, sizeof(int64_t) * E) != cudaSuccess) return FR_ERR_NOMEM;
    if (cudaMalloc(&c->d_new_state_off, sizeof(int64_t) * E) != cudaSuccess) return FR_ERR_NOMEM;
    if (cudaMalloc(&c->d_old_elem_slot, sizeof(int32_t) * E) != cudaSuccess) return FR_ERR_NOMEM;
    if (cudaMalloc(&c->d_old_slot_p, E) != cudaSuccess) return FR_ERR_NOMEM;
    if (cudaMallocHost(&c->h_flag, sizeof(int) * 4) != cudaSuccess) return FR_ERR_NOMEM;
  }
  int* blk_counts = c->d_adapt_i32;
  int* blk_off = blk_counts + nb * (kMaxDeg + 1);
  int* totals = blk_off + nb * (kMaxDeg + 1);
  int32_t* new_slot_elem = totals + (kMaxDeg + 1);
  int32_t* new_elem_slot = new_slot_elem + E;
  int* changed = new_elem_slot + E;
  int8_t* p_old = c->d_adapt_i8;
  int8_t* pa = p_old + E;
  int8_t* pb = pa + E;
  // current degree of every element (host copy is authoritative)
  cudaMemcpyAsync(p_old, c->p.data(), E, cudaMemcpyHostToDevice, s);
  const unsigned ge = (unsigned)((E + 255) / 256);
  FR_LAUNCH(c, "rebucket", s, k_decide<<<ge, 256, 0, s>>>(eta_dev, eta_max_dev, p_old, o->nu_max, o->nu_min,
                                                           o->p_min, o->p_max, E, pa));
  // jump limit: Jacobi sweeps to the fixed point (at most p_max - p_min + 1 rises)
  int sweeps = 0;
  for (;; ++sweeps) {
    if (sweeps > 2 * kMaxDeg + 2) {
      set_error("p_rebucket: neighbour smoothing did not reach its fixed point");
      return FR_ERR_NOT_CONVERGED;
    }
    cudaMemsetAsync(changed, 0, sizeof(int), s);
    FR_LAUNCH(c, "rebucket", s, k_smooth<<<ge, 256, 0, s>>>(pa, c->d_nbr, nf, E, pb, changed));
    cudaMemcpyAsync(c->h_flag, changed, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "p_rebucket");
    std::swap(pa, pb);
    if (c->h_flag[0] == 0) break;
  }
  // stable counting sort by (p, id)
  FR_LAUNCH(c, "rebucket", s, k_sort_count<<<nb, kSortBlock, 0, s>>>(pa, E, blk_counts));
  FR_LAUNCH(c, "rebucket", s, k_sort_scan<<<1, 32, 0, s>>>(blk_counts, nb, blk_off, totals));
  FR_LAUNCH(c, "rebucket", s, k_sort_scatter<<<nb, kSortBlock, 0, s>>>(pa, E, blk_off, new_slot_elem, new_elem_slot));
  FR_LAUNCH(c, "rebucket", s, k_new_offsets<<<ge, 256, 0, s>>>(new_slot_elem, pa, totals, E, c->nd, c->nv,
                                                                c->d_new_state_off));
  // keep the old layout for the transfer
  cudaMemcpyAsync(c->d_old_state_off, c->d_state_off, sizeof(int64_t) * E, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(c->d_old_elem_slot, c->d_elem_slot, sizeof(int32_t) * E, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(c->d_old_slot_p, c->d_slot_p, E, cudaMemcpyDeviceToDevice, s);
  double* xfer = nullptr;
  fr_status e = ensure_transfer_tables(c, &xfer);
  if (e != FR_OK) return e;
  // new degrees to the host (bucket metadata and face lists are rebuilt there)
  std::vector<int8_t> pnew(E);
  cudaMemcpyAsync(pnew.data(), pa, E, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "p_rebucket");
  int64_t ndof_new = 0;
  for (int i = 0; i < E; ++i) {
    const int P = pnew[i] + 1;
    ndof_new += (int64_t)c->nv * (c->nd == 2 ? P * P : P * P * P);
  }
  void* tmp = prec == FR_F64 ? (void*)vec64(c, 10) : (void*)vec32(c, 3);
  if (!tmp) return FR_ERR_NOMEM;
  if (c->nd == 2) {
    if (prec == FR_F64)
      FR_LAUNCH(c, "rebucket", s, k_transfer<double, 2><<<E, 128, 0, s>>>((const double*)q_dev, (double*)tmp, new_slot_elem, c->d_old_elem_slot, c->d_old_state_off, c->d_old_slot_p, pa, c->d_new_state_off, xfer, E));
    else
      FR_LAUNCH(c, "rebucket", s, k_transfer<float, 2><<<E, 128, 0, s>>>((const float*)q_dev, (float*)tmp, new_slot_elem, c->d_old_elem_slot, c->d_old_state_off, c->d_old_slot_p, pa, c->d_new_state_off, xfer, E));
  } else {
    if (prec == FR_F64)
      FR_LAUNCH(c, "rebucket", s, k_transfer<double, 3><<<E, 128, 0, s>>>((const double*)q_dev, (double*)tmp, new_slot_elem, c->d_old_elem_slot, c->d_old_state_off, c->d_old_slot_p, pa, c->d_new_state_off, xfer, E));
    else
      FR_LAUNCH(c, "rebucket", s, k_transfer<float, 3><<<E, 128, 0, s>>>((const float*)q_dev, (float*)tmp, new_slot_elem, c->d_old_elem_slot, c->d_old_state_off, c->d_old_slot_p, pa, c->d_new_state_off, xfer, E));
  }
  const size_t esz = prec == FR_F64 ? 8 : 4;
  cudaMemcpyAsync(q_dev, tmp, esz * ndof_new, cudaMemcpyDeviceToDevice, s);
  if (perm_out_dev) cudaMemcpyAsync(perm_out_dev, new_slot_elem, sizeof(int32_t) * E, cudaMemcpyDeviceToDevice, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check(cudaGetLastError(), "p_rebucket");
  // host metadata: buckets, slot tables and face lists for the new degrees
  const bool same = std::equal(pnew.begin(), pnew.end(), c->p.begin());
  c->p = pnew;
  if (!same) {
    e = build_layout(c);
    if (e != FR_OK) return e;
  }
  return cuda_check(cudaGetLastError(), "p_rebucket");
}

fr_status fr_filter(fr_ctx* c, double* q_dev, double alpha, int32_t p_above, void* stream) {
  if (!c || !q_dev || !(alpha >= 0.0 && alpha <= 1.0)) {
    set_error("fr_filter: bad argument");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  for (const auto& b : c->buckets) {
    if (b.p <= p_above || b.count == 0 || alpha == 0.0) continue;
    const int P = b.p + 1, NSP = c->nd == 2 ? P * P : P * P * P;
    const int64_t nt = (int64_t)b.count * c->nv;
    const unsigned grid = (unsigned)((nt + 127) / 128);
    const double nb = 16.0 * nt * NSP;
#define FILT_CASE(ND, PP) \
  case PP: FR_LAUNCH_B(c, "filter", s, nb, k_filter<ND, PP><<<grid, 128, 0, s>>>((double*)q_dev, c->d_basis64, b.state_base, b.count, alpha)); break;
    if (c->nd == 2) {
      switch (P) { FILT_CASE(2, 2) FILT_CASE(2, 3) FILT_CASE(2, 4) FILT_CASE(2, 5) FILT_CASE(2, 6) }
    } else {
      switch (P) { FILT_CASE(3, 2) FILT_CASE(3, 3) FILT_CASE(3, 4) FILT_CASE(3, 5) FILT_CASE(3, 6) }
    }
#undef FILT_CASE
    (void)NSP;
  }
  return cuda_check(cudaGetLastError(), "fr_filter");
}

fr_status fr_esdirk_tableau(int32_t order, fr_tableau* t) {
  if (!t || (order != 2 && order != 3)) {
    set_error("fr_esdirk_tableau: order must be 2 or 3");
    return FR_ERR_INVALID;
  }
  std::memset(t, 0, sizeof(*t));
  if (order == 2) {
    // 3 stages, stiffly accurate, diagonal g = 1 - sqrt(2)/2, c = (0, 2g, 1)
    const double g = 1.0 - std::sqrt(2.0) / 2.0;
    const double b2 = (0.5 - g) / (2.0 * g), b1 = 1.0 - g - b2;
    t->s = 3;
    const double A[9] = {0, 0, 0, g, g, 0, b1, b2, g};
    std::memcpy(t->A, A, sizeof(A));
    t->b[0] = b1; t->b[1] = b2; t->b[2] = g;
    return FR_OK;
  }
  // 4 stages, order 3, stiffly accurate; g: root of 6g^3 - 18g^2 + 9g - 1 near 0.4359
  double g = 0.44;
  for (int it = 0; it < 60; ++it) g -= (6 * g * g * g - 18 * g * g + 9 * g - 1) / (18 * g * g - 36 * g + 9);
  const double c2 = 2 * g, c3 = 0.6;
  const double r1 = 0.5 - g, r2 = 1.0 / 3.0 - g;
  const double det = c2 * c3 * c3 - c3 * c2 * c2;
  const double b2 = (r1 * c3 * c3 - c3 * r2) / det, b3 = (c2 * r2 - r1 * c2 * c2) / det;
  const double b1 = 1.0 - g - b2 - b3;
  const double a32 = (1.0 / 6.0 - 0.5 * g - 2 * g * g * b2 - g * c3 * b3) / (2 * g * b3);
  const double a31 = c3 - g - a32;
  t->s = 4;
  const double A[16] = {0, 0, 0, 0, g, g, 0, 0, a31, a32, g, 0, b1, b2, b3, g};
  std::memcpy(t->A, A, sizeof(A));
  t->b[0] = b1; t->b[1] = b2; t->b[2] = b3; t->b[3] = g;
  return FR_OK;
}

}  // extern "C"
