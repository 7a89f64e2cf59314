// Element-Jacobi preconditioner of Sec. 2.3: the inverses of the diagonal
// blocks of sigma I - dR/dq, one dense block per element (all of its DOFs),
// applied from the left in GMRES.
//
// Build (once per physical time step in the paper):
//  * the blocks are read off the exact FP32 JVP with unit vectors: elements
//    of one colour of a distance-1 colouring of the face graph are probed
//    together (a face neighbour never shares the colour, so the product
//    restricted to a probed element is that element's own column), one
//    product per colour and local DOF index;
//  * each block sigma I - J_ee is inverted in shared memory by Gauss-Jordan
//    elimination with partial pivoting (FP32), and stored column-major.
// Blocks of up to kPcSmem DOFs are inverted with [A | I] in shared memory;
// larger ones (3D p >= 3: 320, 625 and 1080 DOFs) by a blocked in-place
// Gauss-Jordan elimination on the block in global memory (below).
// Apply: z_e = M_e^-1 (a w_e + b u_e), FP32 arithmetic on FP64 vectors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fr_launch.h"

namespace frgb {

constexpr int kPcSmem = 144;   // largest block inverted in shared memory (2 x 144^2 floats)
constexpr int kPcMax = 1080;   // largest block stored: 3D p = 5 (5 x 216 DOFs)
constexpr int kPanel = 32;     // columns eliminated together by the blocked inversion
constexpr int kTile = 32;      // columns of one tile of the blocked update

static inline int nsp_host(int nd, int p) { return nd == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1); }

// v[state_off(s) + k] = 1 (and the entry k-1 cleared) for slots of colour `col`
__global__ void k_pc_unit(float* __restrict__ v, const int64_t* __restrict__ state_off,
                          const int32_t* __restrict__ slot_color, int slot_begin, int count, int nb, int col,
                          int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int s = slot_begin + i;
  if (slot_color[s] != col) return;
  if (k > 0 && k - 1 < nb) v[state_off[s] + k - 1] = 0.0f;
  if (k < nb) v[state_off[s] + k] = 1.0f;
}

// column k of B_s = sigma I - J_ss (column-major, B[k * nb + i]) for slots of colour `col`
__global__ void k_pc_gather(float* __restrict__ B, const int64_t* __restrict__ pc_off, const float* __restrict__ J,
                            const int64_t* __restrict__ state_off, const int32_t* __restrict__ slot_color,
                            int slot_begin, int count, int nb, int col, int k, float sigma) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * nb) return;
  const int i = (int)(t % nb);
  const int s = slot_begin + (int)(t / nb);
  if (slot_color[s] != col || pc_off[s] < 0) return;
  const float val = (i == k ? sigma : 0.0f) - J[state_off[s] + i];
  B[pc_off[s] + (int64_t)k * nb + i] = val;
}

// In-place inverse of one nb x nb block per CTA (column-major in global
// memory) by Gauss-Jordan elimination on [A | I] in shared memory, partial
// pivoting by rows.  A zero pivot sets *status and leaves the block as is.
__global__ void k_pc_invert(float* __restrict__ B, const int64_t* __restrict__ pc_off, int slot_begin, int nb,
                            int* __restrict__ status) {
  extern __shared__ __align__(16) float sm[];
  float* M = sm;                    // [nb][2 nb] row-major
  __shared__ float pv[32];
  __shared__ int pr[32];
  __shared__ int piv;
  const int s = slot_begin + blockIdx.x;
  const int64_t off = pc_off[s];
  if (off < 0) return;
  float* A = B + off;
  const int w2 = 2 * nb;
  for (int t = threadIdx.x; t < nb * w2; t += blockDim.x) {
    const int r = t / w2, cidx = t % w2;
    M[t] = cidx < nb ? A[(int64_t)cidx * nb + r] : (cidx - nb == r ? 1.0f : 0.0f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int k = 0; k < nb; ++k) {
    // pivot: the row r >= k with the largest |M[r][k]| (lowest row at a tie)
    float best = -1.0f;
    int br = k;
    for (int r = k + threadIdx.x; r < nb; r += blockDim.x) {
      const float a = fabsf(M[r * w2 + k]);
      if (a > best) {
        best = a;
        br = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_down_sync(0xffffffffu, best, o);
      const int orr = __shfl_down_sync(0xffffffffu, br, o);
      if (ob > best || (ob == best && orr < br)) {
        best = ob;
        br = orr;
      }
    }
    if (lane == 0) {
      pv[warp] = best;
      pr[warp] = br;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float b0 = pv[0];
      int r0 = pr[0];
      for (int q = 1; q < nw; ++q)
        if (pv[q] > b0 || (pv[q] == b0 && pr[q] < r0)) {
          b0 = pv[q];
          r0 = pr[q];
        }
      piv = (b0 > 0.0f) ? r0 : -1;
      if (piv < 0) atomicExch(status, 1);
    }
    __syncthreads();
    if (piv < 0) return;   // singular block: reported through status
    if (piv != k)
      for (int cidx = threadIdx.x; cidx < w2; cidx += blockDim.x) {
        const float a = M[k * w2 + cidx];
        M[k * w2 + cidx] = M[piv * w2 + cidx];
        M[piv * w2 + cidx] = a;
      }
    __syncthreads();
    const float inv = 1.0f / M[k * w2 + k];
    __syncthreads();
    for (int cidx = threadIdx.x; cidx < w2; cidx += blockDim.x) M[k * w2 + cidx] *= inv;
    __syncthreads();
    // eliminate column k from every other row (the factors read before any row changes)
    for (int t = threadIdx.x; t < nb * w2; t += blockDim.x) {
      const int r = t / w2, cidx = t % w2;
      if (r == k || cidx == k) continue;
      M[t] -= M[r * w2 + k] * M[k * w2 + cidx];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nb; r += blockDim.x)
      if (r != k) M[r * w2 + k] = 0.0f;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t % nb, cidx = t / nb;   // column-major output
    A[(int64_t)cidx * nb + r] = M[r * w2 + nb + cidx];
  }
}

// In-place inverse of one nb x nb block per CTA (column-major in global
// memory) by Gauss-Jordan elimination with partial pivoting, blocked by
// panels of kPanel columns: each panel is eliminated in shared memory (pivot
// search over the rows not yet used, row swaps, scaling, elimination from
// every other row), and its kPanel pivots then reach every other column at
// once as the panel's row permutation followed by the rank-kPanel update
// A[:, j] += (panel - I) A[K, j]; the row swaps are undone as column swaps at
// the end.  The block moves through global memory (L2) once per panel, and the
// nb^3 multiply-adds of the inversion are register-tiled in the update.  A
// zero pivot sets *status and leaves the block unfinished.
// Shared memory: the panel [nb][kPanel + 1], the panel's row order idx[nb],
// the pivot rows perm[nb], the pivot column fcol[nb], the pivot row rk[kPanel],
// the tile's panel rows X[kPanel][kTile + 1] and permuted rows [2 kPanel][kTile].
__global__ void __launch_bounds__(512) k_pc_invert_blocked(float* __restrict__ B, const int64_t* __restrict__ pc_off,
                                                           int slot_begin, int nb, int* __restrict__ status) {
  extern __shared__ __align__(16) float sm[];
  constexpr int LD = kPanel + 1;
  float* Pn = sm;                                   // [nb][LD]
  float* fcol = Pn + (size_t)nb * LD;               // [nb]
  float* X = fcol + nb;                             // [kPanel][kTile + 1]
  float* Y = X + kPanel * (kTile + 1);              // [2 kPanel][kTile]
  float* rk = Y + 2 * kPanel * kTile;               // [kPanel]
  int* idx = reinterpret_cast<int*>(rk + kPanel);   // [nb]
  int* perm = idx + nb;                             // [nb]
  __shared__ float pv[16];
  __shared__ int pr[16];
  __shared__ int piv;
  const int s = slot_begin + blockIdx.x;
  const int64_t off = pc_off[s];
  if (off < 0) return;
  float* A = B + off;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int kb = 0; kb < nb; kb += kPanel) {
    const int nk = min(kPanel, nb - kb);
    // panel in shared memory; its row order starts as the identity
    for (int t = tid; t < nb * nk; t += nt) {
      const int c = t / nb, r = t % nb;
      Pn[r * LD + c] = A[(int64_t)(kb + c) * nb + r];
    }
    for (int r = tid; r < nb; r += nt) idx[r] = r;
    __syncthreads();
    for (int kl = 0; kl < nk; ++kl) {
      const int k = kb + kl;
      // pivot: the row r >= k with the largest |Pn[r][kl]| (lowest row at a tie)
      float best = -1.0f;
      int br = k;
      for (int r = k + tid; r < nb; r += nt) {
        const float a = fabsf(Pn[r * LD + kl]);
        if (a > best) {
          best = a;
          br = r;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_down_sync(0xffffffffu, best, o);
        const int orr = __shfl_down_sync(0xffffffffu, br, o);
        if (ob > best || (ob == best && orr < br)) {
          best = ob;
          br = orr;
        }
      }
      if (lane == 0) {
        pv[warp] = best;
        pr[warp] = br;
      }
      __syncthreads();
      if (tid == 0) {
        float b0 = pv[0];
        int r0 = pr[0];
        for (int q = 1; q < nw; ++q)
          if (pv[q] > b0 || (pv[q] == b0 && pr[q] < r0)) {
            b0 = pv[q];
            r0 = pr[q];
          }
        piv = (b0 > 0.0f) ? r0 : -1;
        if (piv < 0) atomicExch(status, 1);
        else perm[k] = r0;
      }
      __syncthreads();
      const int p = piv;
      if (p < 0) return;   // singular block: reported through status
      if (p != k) {
        for (int c = tid; c < nk; c += nt) {
          const float a = Pn[k * LD + c];
          Pn[k * LD + c] = Pn[p * LD + c];
          Pn[p * LD + c] = a;
        }
        if (tid == 0) {
          const int t0 = idx[k];
          idx[k] = idx[p];
          idx[p] = t0;
        }
      }
      __syncthreads();
      const float inv = 1.0f / Pn[k * LD + kl];
      for (int r = tid; r < nb; r += nt) fcol[r] = Pn[r * LD + kl];
      for (int c = tid; c < nk; c += nt) rk[c] = c == kl ? inv : Pn[k * LD + c] * inv;
      __syncthreads();
      for (int t = tid; t < nb * nk; t += nt) {
        const int r = t / nk, c = t % nk;
        if (r == k) Pn[r * LD + c] = rk[c];
        else if (c == kl) Pn[r * LD + c] = -fcol[r] * inv;
        else Pn[r * LD + c] -= fcol[r] * rk[c];
      }
      __syncthreads();
    }
    // the eliminated panel back to global memory
    for (int t = tid; t < nb * nk; t += nt) {
      const int c = t / nb, r = t % nb;
      A[(int64_t)(kb + c) * nb + r] = Pn[r * LD + c];
    }
    // every other column j: rows permuted as the panel's were, then
    // A[:, j] += (Pn - I_K) A[K, j]
    const int tx = tid % (kTile / 4), ty = tid / (kTile / 4), nty = nt / (kTile / 4);
    for (int j0 = 0; j0 < nb; j0 += kTile) {
      // columns j0 .. j0 + kTile - 1 that lie outside the panel
      __syncthreads();
      // (a) row permutation of the tile: the rows that can have moved are the
      // panel rows and their pivot rows (all reads before any write)
      for (int t = tid; t < 2 * nk * kTile; t += nt) {
        const int ri = t / kTile, c = t % kTile, j = j0 + c;
        const int r = ri < nk ? kb + ri : perm[kb + ri - nk];
        if (j < nb && (j < kb || j >= kb + nk)) Y[ri * kTile + c] = A[(int64_t)j * nb + idx[r]];
      }
      __syncthreads();
      for (int t = tid; t < 2 * nk * kTile; t += nt) {
        const int ri = t / kTile, c = t % kTile, j = j0 + c;
        const int r = ri < nk ? kb + ri : perm[kb + ri - nk];
        if (j < nb && (j < kb || j >= kb + nk)) A[(int64_t)j * nb + r] = Y[ri * kTile + c];
      }
      __syncthreads();
      // (b) the panel rows of the tile
      for (int t = tid; t < nk * kTile; t += nt) {
        const int k = t / kTile, c = t % kTile, j = j0 + c;
        X[k * (kTile + 1) + c] = (j < nb && (j < kb || j >= kb + nk)) ? A[(int64_t)j * nb + kb + k] : 0.0f;
      }
      __syncthreads();
      // (c) rank-nk update, four rows x four columns a thread per step
      for (int r0 = ty; r0 < nb; r0 += 4 * nty) {
        float acc[4][4];
        int rows[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          rows[m] = r0 + m * nty;
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[m][c] = 0.0f;
        }
        for (int k = 0; k < nk; ++k) {
          float x[4], w[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) x[c] = X[k * (kTile + 1) + tx * 4 + c];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int r = rows[m];
            w[m] = r < nb ? Pn[r * LD + k] - (r == kb + k ? 1.0f : 0.0f) : 0.0f;
          }
#pragma unroll
          for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[m][c] = fmaf(w[m], x[c], acc[m][c]);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int r = rows[m];
          if (r >= nb) continue;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int j = j0 + tx * 4 + c;
            if (j < nb && (j < kb || j >= kb + nk)) A[(int64_t)j * nb + r] += acc[m][c];
          }
        }
      }
    }
    __syncthreads();
  }
  // undo the row swaps as column swaps, last pivot first
  for (int k = nb - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int r = tid; r < nb; r += nt) {
        const float a = A[(int64_t)k * nb + r];
        A[(int64_t)k * nb + r] = A[(int64_t)p * nb + r];
        A[(int64_t)p * nb + r] = a;
      }
    __syncthreads();
  }
}

static size_t pc_blocked_smem(int nb) {
  return sizeof(float) * ((size_t)nb * (kPanel + 1) + nb + kPanel * (kTile + 1) + 2 * kPanel * kTile + kPanel) +
         sizeof(int) * 2 * (size_t)nb;
}

// z_e = M_e^-1 (a w_e + b u_e) for blocks of more than 256 rows: one CTA per
// element, the rows strided over its threads (coalesced column-major reads).
// The vectors are FP64 or FP32 (VT; the FP32 Krylov basis), the sums FP32.
template <typename VT>
__global__ void __launch_bounds__(256) k_pc_apply_big(const float* __restrict__ B, const int64_t* __restrict__ pc_off,
                                                      const int64_t* __restrict__ state_off, int slot_begin, int nb,
                                                      double a, const VT* w, double b,
                                                      const VT* __restrict__ u, VT* z, double inv_sigma,
                                                      const int* __restrict__ gate, const double* __restrict__ bscale) {
  extern __shared__ __align__(16) float xs[];   // [nb]
  if (gate && *gate) return;
  if (bscale) b *= *bscale;
  const int s = slot_begin + blockIdx.x;
  const int64_t base = state_off[s], off = pc_off[s];
  double xv[kPcMax / 256 + 1];
  int nr = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x, ++nr) {
    xv[nr] = a * (double)w[base + i] + (u ? b * (double)u[base + i] : 0.0);
    xs[i] = (float)xv[nr];
  }
  __syncthreads();
  nr = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x, ++nr) {
    if (off < 0) {
      z[base + i] = (VT)(xv[nr] * inv_sigma);
      continue;
    }
    const float* Bc = B + off;
    float acc = 0.0f;
    for (int j = 0; j < nb; ++j) acc = fmaf(Bc[(int64_t)j * nb + i], xs[j], acc);
    z[base + i] = (VT)acc;
  }
}

// z_e = M_e^-1 (a w_e + b u_e); epb elements per CTA, one thread per row.
// Elements without a stored block (pc_off < 0): z_e = (a w_e + b u_e) / sigma.
template <typename VT>
__global__ void k_pc_apply(const float* __restrict__ B, const int64_t* __restrict__ pc_off,
                           const int64_t* __restrict__ state_off, int slot_begin, int count, int nb, int epb,
                           double a, const VT* w, double b, const VT* __restrict__ u, VT* z,
                           double inv_sigma, const int* __restrict__ gate, const double* __restrict__ bscale) {
  extern __shared__ __align__(16) float xs[];   // [epb][nb]
  if (gate && *gate) return;
  if (bscale) b *= *bscale;
  const int le = threadIdx.x / nb, i = threadIdx.x % nb;
  const int e = blockIdx.x * epb + le;
  const bool valid = le < epb && e < count;
  int64_t base = 0, off = -1;
  double x = 0.0;
  if (valid) {
    const int s = slot_begin + e;
    base = state_off[s];
    off = pc_off[s];
    x = a * (double)w[base + i] + (u ? b * (double)u[base + i] : 0.0);
    xs[le * nb + i] = (float)x;
  }
  __syncthreads();
  if (!valid) return;
  if (off < 0) {
    z[base + i] = (VT)(x * inv_sigma);
    return;
  }
  const float* Bc = B + off;
  const float* xe = xs + le * nb;
  float acc = 0.0f;
  for (int j = 0; j < nb; ++j) acc = fmaf(Bc[(int64_t)j * nb + i], xe[j], acc);
  z[base + i] = (VT)acc;
}

// z = (a w + b u) / sigma on every DOF of a bucket without stored blocks
template <typename VT>
__global__ void k_pc_scale(const int64_t* __restrict__ state_off, int slot_begin, int count, int nb, double a,
                           const VT* w, double b, const VT* __restrict__ u, VT* z, double inv_sigma,
                           const int* __restrict__ gate, const double* __restrict__ bscale) {
  if (gate && *gate) return;
  if (bscale) b *= *bscale;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * nb) return;
  const int64_t idx = state_off[slot_begin + (int)(t / nb)] + (int)(t % nb);
  z[idx] = (VT)((a * (double)w[idx] + (u ? b * (double)u[idx] : 0.0)) * inv_sigma);
}

// Distance-1 colouring of the face graph (greedy in element order), once per context.
void pc_color(fr_ctx* c) {
  const int E = c->E, nf = c->nf;
  c->color.assign(E, -1);
  int nc = 0;
  std::vector<char> used;
  for (int e = 0; e < E; ++e) {
    used.assign(nc + 1, 0);
    for (int f = 0; f < nf; ++f) {
      const int n = c->nbr[(size_t)e * nf + f];
      if (n >= 0 && n != e && c->color[n] >= 0) used[c->color[n]] = 1;
    }
    int col = 0;
    while (col < nc && used[col]) ++col;
    c->color[e] = col;
    nc = std::max(nc, col + 1);
  }
  c->n_colors = nc;
}

}  // namespace frgb

using namespace frgb;

extern "C" {

fr_status fr_precond_build(fr_ctx* c, const double* q64_dev, double sigma, void* stream) {
  if (!c || !q64_dev || !(sigma > 0.0)) {
    set_error("fr_precond_build: bad argument");
    return FR_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int E = c->E, nd = c->nd, nv = c->nv;
  if (c->color.empty()) pc_color(c);
  // block offsets per slot (floats), -1 for blocks larger than kPcMax
  std::vector<int64_t> off(E, -1);
  std::vector<int32_t> slot_color(E);
  int64_t total = 0;
  int kmax = 0;
  for (const auto& b : c->buckets) {
    const int nb = nv * nsp_host(nd, b.p);
    for (int i = 0; i < b.count; ++i) {
      const int sl = b.slot_begin + i;
      slot_color[sl] = c->color[c->slot_elem[sl]];
      if (nb <= kPcMax) {
        off[sl] = total;
        total += (int64_t)nb * nb;
      }
    }
    if (nb <= kPcMax && b.count > 0) kmax = std::max(kmax, nb);
  }
  if (!c->d_pc_off && cudaMalloc(&c->d_pc_off, sizeof(int64_t) * E) != cudaSuccess) return FR_ERR_NOMEM;
  if (!c->d_slot_color && cudaMalloc(&c->d_slot_color, sizeof(int32_t) * E) != cudaSuccess) return FR_ERR_NOMEM;
  if (total > c->pc_cap) {
    cudaFree(c->d_pc);
    c->d_pc = nullptr;
    c->pc_cap = 0;
    if (cudaMalloc(&c->d_pc, sizeof(float) * std::max<int64_t>(total, 1)) != cudaSuccess) {
      cudaGetLastError();
      set_error("fr_precond_build: block storage allocation failed");
      return FR_ERR_NOMEM;
    }
    c->pc_cap = total;
  }
  if (!c->d_pc_status && cudaMalloc(&c->d_pc_status, sizeof(int)) != cudaSuccess) return FR_ERR_NOMEM;
  cudaMemcpyAsync(c->d_pc_off, off.data(), sizeof(int64_t) * E, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(c->d_slot_color, slot_color.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(c->d_pc_status, 0, sizeof(int), s);
  c->pc_ready = false;
  const int64_t n = c->n_dof;
  float* q32 = vec32(c, 0);
  float* v32 = vec32(c, 1);
  float* J32 = vec32(c, 2);
  if (!q32 || !v32 || !J32) return FR_ERR_NOMEM;
  vcast_f64_f32(c, q64_dev, q32, n, s);
  fr_status e = launch_jvp_prepare(c, q32, FR_F32, s);
  if (e != FR_OK) return e;
  const float sg = (float)sigma;
  for (int col = 0; col < c->n_colors && kmax > 0; ++col) {
    cudaMemsetAsync(v32, 0, sizeof(float) * n, s);
    for (int k = 0; k < kmax; ++k) {
      for (const auto& b : c->buckets) {
        const int nb = nv * nsp_host(nd, b.p);
        if (nb > kPcMax) continue;
        FR_LAUNCH(c, "precond_build", s,
                  k_pc_unit<<<(b.count + 255) / 256, 256, 0, s>>>(v32, c->d_state_off, c->d_slot_color,
                                                                  b.slot_begin, b.count, nb, col, k));
      }
      if ((e = launch_jvp_prepared(c, q32, v32, J32, FR_F32, s)) != FR_OK) return e;
      for (const auto& b : c->buckets) {
        const int nb = nv * nsp_host(nd, b.p);
        if (nb > kPcMax || k >= nb) continue;
        const int64_t nt = (int64_t)b.count * nb;
        FR_LAUNCH(c, "precond_build", s,
                  k_pc_gather<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(c->d_pc, c->d_pc_off, J32, c->d_state_off,
                                                                          c->d_slot_color, b.slot_begin, b.count, nb,
                                                                          col, k, sg));
      }
    }
  }
  for (const auto& b : c->buckets) {
    const int nb = nv * nsp_host(nd, b.p);
    if (nb > kPcMax || b.count == 0) continue;
    if (nb <= kPcSmem) {
      const size_t smem = sizeof(float) * 2 * (size_t)nb * nb;
      cudaFuncSetAttribute(k_pc_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      FR_LAUNCH(c, "precond_build", s,
                k_pc_invert<<<b.count, 256, smem, s>>>(c->d_pc, c->d_pc_off, b.slot_begin, nb, c->d_pc_status));
    } else {
      const size_t smem = pc_blocked_smem(nb);
      cudaFuncSetAttribute(k_pc_invert_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      FR_LAUNCH(c, "precond_build", s,
                k_pc_invert_blocked<<<b.count, 512, smem, s>>>(c->d_pc, c->d_pc_off, b.slot_begin, nb,
                                                               c->d_pc_status));
    }
  }
  int status = 0;
  cudaMemcpyAsync(&status, c->d_pc_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  fr_status st = cuda_check(cudaStreamSynchronize(s), "fr_precond_build");
  if (st != FR_OK) return st;
  if (status) {
    set_error("fr_precond_build: singular element block");
    return FR_ERR_NONFINITE;
  }
  c->pc_sigma = sigma;
  c->pc_ready = true;
  return FR_OK;
}

fr_status fr_precond_release(fr_ctx* c) {
  if (!c) return FR_ERR_INVALID;
  cudaFree(c->d_pc);
  c->d_pc = nullptr;
  c->pc_cap = 0;
  c->pc_ready = false;
  return FR_OK;
}

}  // extern "C"

namespace frgb {

// z = M^-1 (a w + b u) on every element (z may alias w)
template <typename VT>
static fr_status precond_apply_t(fr_ctx* c, double a, const VT* w, double b, const VT* u, VT* z, cudaStream_t s,
                                 const int* gate, const double* bscale) {
  if (!c->pc_ready) {
    set_error("element-Jacobi preconditioner not built (fr_precond_build) for the current layout");
    return FR_ERR_INVALID;
  }
  const int nd = c->nd, nv = c->nv;
  const double vb = 3.0 * sizeof(VT);   // a w, b u in, z out
  for (const auto& bk : c->buckets) {
    if (bk.count == 0) continue;
    const int nb = nv * nsp_host(nd, bk.p);
    if (nb > kPcMax) {   // no stored blocks in this bucket: 1/sigma
      const int64_t nt = (int64_t)bk.count * nb;
      FR_LAUNCH_B(c, "precond_apply", s, vb * nt,
                  k_pc_scale<VT><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(c->d_state_off, bk.slot_begin, bk.count,
                                                                            nb, a, w, b, u, z, 1.0 / c->pc_sigma,
                                                                            gate, bscale));
      continue;
    }
    const double bytes = (double)bk.count * nb * (vb + 4.0 * nb);
    if (nb > 256) {
      FR_LAUNCH_B(c, "precond_apply", s, bytes,
                  k_pc_apply_big<VT><<<bk.count, 256, sizeof(float) * nb, s>>>(c->d_pc, c->d_pc_off, c->d_state_off,
                                                                               bk.slot_begin, nb, a, w, b, u, z,
                                                                               1.0 / c->pc_sigma, gate, bscale));
      continue;
    }
    const int epb = 256 / nb;
    const int threads = epb * nb;
    const unsigned grid = (unsigned)((bk.count + epb - 1) / epb);
    FR_LAUNCH_B(c, "precond_apply", s, bytes,
                k_pc_apply<VT><<<grid, threads, sizeof(float) * threads, s>>>(c->d_pc, c->d_pc_off, c->d_state_off,
                                                                              bk.slot_begin, bk.count, nb, epb, a, w,
                                                                              b, u, z, 1.0 / c->pc_sigma, gate,
                                                                              bscale));
  }
  return cuda_check(cudaGetLastError(), "precond_apply");
}

fr_status precond_apply(fr_ctx* c, double a, const double* w, double b, const double* u, double* z, cudaStream_t s,
                        const int* gate, const double* bscale) {
  return precond_apply_t<double>(c, a, w, b, u, z, s, gate, bscale);
}

fr_status precond_apply(fr_ctx* c, double a, const float* w, double b, const float* u, float* z, cudaStream_t s,
                        const int* gate, const double* bscale) {
  return precond_apply_t<float>(c, a, w, b, u, z, s, gate, bscale);
}

}  // namespace frgb

extern "C" fr_status fr_precond_apply(fr_ctx* c, const double* w_dev, double* z_dev, void* stream) {
  if (!c || !w_dev || !z_dev) {
    set_error("fr_precond_apply: null argument");
    return FR_ERR_INVALID;
  }
  return precond_apply(c, 1.0, w_dev, 0.0, nullptr, z_dev, (cudaStream_t)stream);
}
