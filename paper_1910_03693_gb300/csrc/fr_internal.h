// Internal declarations of the GB300 FR library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fr.h"
#include "timing.h"

namespace frgb {

constexpr int kMaxDeg = 5;   // highest polynomial degree supported
constexpr int kPM = 6;       // most solution points per direction (kMaxDeg + 1)

// 1D operators of one degree (P = p + 1 Gauss-Legendre points), Sec. 2.2.
template <typename T>
struct BasisTab {
  T x[kPM], w[kPM];
  T D[kPM][kPM];        // D[i][k] = l_k'(x_i)
  T ext[2][kPM];        // l_k(-1), l_k(+1)
  T dext[2][kPM];       // l_k'(-1), l_k'(+1)
  T dg[2][kPM];         // g_L'(x_i), g_R'(x_i) of the DG (Radau) correction functions
  T dgf[2];             // g_L'(-1) = -(p+1)^2/2, g_R'(+1) = (p+1)^2/2
  T modal[kPM][kPM];    // Legendre coefficients c_m = sum_i modal[m][i] s_i
  T nodal[kPM][kPM];    // s_i = sum_m nodal[i][m] c_m  (nodal[i][m] = P_m(x_i))
  T Dh[kPM][kPM];       // D - g_L' (x) l(-1) - g_R' (x) l(+1): derivative with the local
                        // end values removed, so div = Dh F + g_L' F^com_L + g_R' F^com_R
};

// Mortar operators from Ps slave points to Pm mortar points and back.
template <typename T>
struct MortarTab {
  T I[kPM][kPM];        // I[m][a] = l_a^{slave}(x_m^{mortar})
  T Pi[kPM][kPM];       // Pi[a][m] = w_m l_a(x_m) / w_a  (L2 projection)
};

// Host construction of the tables (basis.cpp).
void build_basis(int p, BasisTab<double>& t);
void build_mortar(int ps, int pm, MortarTab<double>& t);
void lagrange_eval(const double* xs, int n, double x, double* out);
void lagrange_deriv_eval(const double* xs, int n, double x, double* out);
void gauss_legendre(int P, double* x, double* w);
double legendre_p(int n, double x);

// Face records.  Offsets are absolute element-face block starts in the
// trace (t) and face-output (o) workspaces.
struct FaceRec {
  int64_t mt, st, mo, so;
  int32_t me, se;      // element ids (geometry lookup)
  int32_t mf, sf;      // face indices
  int32_t orient, idx; // master's orientation code; index of the face in its group
};
struct BndRec {
  int64_t mt, mo;
  int32_t me, mf;
};

// Strided view of the geometry: metric terms S[d][j] (k = d*nd + j), |J|
// (k = nd*nd) and 1/|J| (k = nd*nd + 1) at solution and face points; at face
// points also |S_d| (k = nd*nd + 2 + d) and 1/|S_d| (k = nd*nd + 2 + nd + d),
// S_d the row d of S (the face area vector of a face normal to axis d).
// Everything that does not depend on the state is computed once on the host
// in FP64: the FP64 divides and square roots it saves are expensive on GB300.
inline int geo_nk_vol(int nd) { return nd * nd + 2; }
inline int geo_nk_face(int nd) { return nd * nd + 2 + 2 * nd; }
template <typename T>
struct GeoView {
  const T* vol;         // value(e, k, sp) = vol[e*ves + k*vks + sp*vps]
  int64_t ves;
  int32_t vks, vps;
  const T* face;        // value(e, f, k, t) = face[e*fes + f*ffs + k*fks + t*fps]
  int64_t fes;
  int32_t ffs, fks, fps;
};

struct Bucket {
  int p = 0, count = 0, slot_begin = 0;
  int64_t state_base = 0;   // values
  int64_t trace_base = 0;   // values
  int64_t out_base = 0;     // values
  int64_t ctrace_base = 0;  // values: compact traces of the fused JVP (q and its normal derivative)
};

struct FaceGroup {
  int pm = 0, ps = 0, n = 0;
  FaceRec* d_recs = nullptr;
  int64_t scratch_base = 0; // values, mixed-degree groups only
};
struct BndGroup {
  int p = 0, kind = 0, n = 0;
  BndRec* d_recs = nullptr;
};

// One tile of elements of one bucket: the unit of the multi-bucket launch.
struct WorkItem {
  int32_t bucket;   // index into the launch's bucket table
  int32_t first;    // first element (bucket-local)
};

// Neighbour of one element face for the fused JVP (slot-major, face-minor).
struct FusedNbr {
  int32_t nloc;    // the neighbour's bucket-local index (conforming faces: the same bucket)
  int32_t nelem;   // the neighbour's element id (its geometry)
  int32_t g;       // the neighbour's face
  int32_t code;    // bits 0-7: orientation code (this side's point -> the neighbour's); bit 8: this side is the master
};

// Elements per tile of the multi-bucket launch: as many as fill a 256-thread block.
inline int epb_multi(int nd, int P) {
  const int nsp = nd == 2 ? P * P : P * P * P;
  return nsp >= 256 ? 1 : 256 / nsp;
}

// Element weight of the multi-bucket work table (tuning slot [0][0][P = 1]):
// 0 n_sp (p+1) (the default), 1 n_sp, 2 n_sp^2, 3 n_sp^3 -- the paper's
// candidate element weights for repartitioning (Sec. 3.2), reused as CTA
// work weights for the order in which the persistent launch takes tiles.
inline double element_weight(int model, int nsp, int P) {
  switch (model) {
    case 1: return (double)nsp;
    case 2: return (double)nsp * nsp;
    case 3: return (double)nsp * nsp * nsp;
    default: return (double)nsp * P;
  }
}

struct PhysParams {
  double gamma, mu, Pr, kappa;
  double q_inf[5];
  int flux;   // FR_FLUX_RUSANOV or FR_FLUX_ROE
};

}  // namespace frgb

struct fr_ctx {
  int nd = 0, nv = 0, nf = 0, E = 0, geom_order = 1, p_min = 1, p_max = 1;
  bool affine = false, visc = false;
  bool diag_mesh = false;   // 3D, affine, every metric diagonal (axis-aligned boxes)
  bool diag = false;        // diag_mesh and the diagonal-metric kernels enabled
  frgb::PhysParams phys{};
  int device = 0;
  // host mesh
  std::vector<double> nodes;
  std::vector<int32_t> nbr;
  std::vector<int8_t> nbr_face, orient, p;
  // tables (device)
  frgb::BasisTab<double>* d_basis64 = nullptr;   // [kPM + 1], indexed by P
  frgb::BasisTab<float>* d_basis32 = nullptr;
  frgb::BasisTab<float>* d_basis16 = nullptr;    // operators rounded to bfloat16 (FR_BF16OP)
  frgb::MortarTab<double>* d_mortar64 = nullptr; // [(kPM+1)*(kPM+1)], index Pm*(kPM+1)+Ps
  frgb::MortarTab<float>* d_mortar32 = nullptr;
  frgb::MortarTab<float>* d_mortar16 = nullptr;
  bool bf16op = false;      // FP32 kernels read the bfloat16-rounded operators
  // geometry (device): affine -> per element constants; else per degree
  double* d_gaff64 = nullptr;
  float* d_gaff32 = nullptr;
  double* d_gvol64[frgb::kMaxDeg + 1] = {};
  float* d_gvol32[frgb::kMaxDeg + 1] = {};
  double* d_gface64[frgb::kMaxDeg + 1] = {};
  float* d_gface32[frgb::kMaxDeg + 1] = {};
  // double-float copies of the tables, created on the first FR_DF residual
  // (type frgb::dfloat, 8 bytes a value)
  void* d_basis_df = nullptr;
  void* d_mortar_df = nullptr;
  void* d_gaff_df = nullptr;
  void* d_gvol_df[frgb::kMaxDeg + 1] = {};
  void* d_gface_df[frgb::kMaxDeg + 1] = {};
  bool df_ready = false;
  // layout
  std::vector<frgb::Bucket> buckets;     // one per degree present, ascending p
  std::vector<int32_t> slot_elem;        // bucket position -> element id
  int64_t n_dof = 0, n_dof_cap = 0;
  int32_t* d_slot_elem = nullptr;        // [E]
  int64_t* d_canon_off = nullptr;        // [E] canonical offset of the element at each slot
  int64_t* d_state_off = nullptr;        // [E] state offset of the element at each slot
  int8_t* d_slot_p = nullptr;            // [E] degree at each slot
  int32_t* d_elem_slot = nullptr;        // [E] slot of each element
  // workspaces (bytes sized for FP64 at capacity)
  int nvt = 0;                           // trace components per face point
  int64_t trace_cap = 0, fout_cap = 0, scratch_cap = 0;
  void* d_trace_q = nullptr;
  void* d_trace_v = nullptr;
  void* d_fout = nullptr;
  void* d_scratch = nullptr;
  void* d_fbar = nullptr;                // VJP: adjoints of the face outputs
  void* d_trbar = nullptr;               // VJP: adjoints of the traces
  // faces
  std::vector<frgb::FaceGroup> fgroups;
  std::vector<frgb::BndGroup> bgroups;
  int32_t* d_nbr = nullptr;              // [E][nf] for the adaptation smoother
  // solver workspaces (lazily allocated)
  double* d_krylov = nullptr;
  double* d_step = nullptr;              // esdirk_step: stage residuals, q^n, stage value, eta
  // element-Jacobi preconditioner (left): inverse blocks in slot order, column-major
  std::vector<int> color;                // distance-1 colouring of the face graph (element id)
  int n_colors = 0;
  float* d_pc = nullptr;
  int64_t pc_cap = 0;                    // floats in d_pc
  int64_t* d_pc_off = nullptr;           // [E] block offset of each slot, -1 = no block (1/sigma)
  int32_t* d_slot_color = nullptr;       // [E] colour of each slot
  int* d_pc_status = nullptr;
  bool pc_ready = false;
  double pc_sigma = 0.0;
  int64_t step_cap = 0;                  // doubles in d_step            // (m+1) * n_dof_cap basis
  int krylov_m = 0;
  float* d_krylov32 = nullptr;            // the FP32 Krylov basis ((m+1) * ld), when used
  int krylov32_m = 0;
  bool f32_basis = true;                 // GMRES with FP32 products: FP32 Krylov basis
  double* d_vec64[13] = {};   // 0-2 FD Jv, 3 Jv, 4-5 GMRES, 6-9 ESDIRK, 10-11 adaptation, 12 host staging
  float* d_vec32[4] = {};
  double* d_red = nullptr;               // reduction scratch
  int64_t red_cap = 0;
  double* h_red = nullptr;               // pinned host mirror
  frgb::Timing timing;                   // launch counter and optional per-kernel events
  // launch configuration: elements per CTA by [precision][kind][P] (kind 0
  // trace, 1 volume residual, 2 volume JVP), 0 = default; cost-ordered work
  // tables of the multi-bucket launch by (precision, kind)
  int epb_tab[2][3][frgb::kPM + 1] = {};
  bool multi_launch = true;
  // work table of the multi-bucket launch (the same for every precision and
  // kernel kind), rebuilt eagerly whenever the layout or the weight model
  // changes, so that no launch ever allocates it
  frgb::WorkItem* d_work = nullptr;
  int n_work = 0;
  // fused JVP: every face interior and conforming (then the exact JVP runs as
  // compact traces + one face-and-volume kernel); the neighbour of every
  // element face, slot-major (frgb::FusedNbr)
  bool fused_ok = false;
  bool use_fused = true;
  void* d_fnbr = nullptr;
  // CUDA graph of one Arnoldi matrix-vector product -J(q) V[j] (per precision),
  // with the column index read from d_jidx; keyed by the pointers it captured
  cudaGraphExec_t jvp_graph[2] = {nullptr, nullptr};
  const void* jvp_graph_key[2][5] = {};
  int jvp_graph_nodes[2] = {0, 0};
  std::vector<frgb::TimerRec> graph_timers[2];  // event pairs inside each graph
  bool graph_timers_live[2] = {false, false};   // a replay's timers are not yet accumulated
  bool use_graphs = true;
  bool use_diag = true;
  bool df_arnoldi = false;    // Arnoldi dot products in double-float arithmetic (FP32 pipe)
  int arnoldi_map = 1;        // slot walk of the Arnoldi reductions (0 grid-strided, 1 warp runs)
  bool use_tma = true;        // compact face kernel staged by bulk asynchronous copies where it can be
  int* d_status = nullptr;    // device status word: bit 0, a bounded wait of a kernel gave up
  // device-driven GMRES cycles (exact products): the gate word the cycle's
  // Arnoldi launches read (non-null only while such a cycle launches them;
  // see gate_closed), the cycle's Hessenberg columns, rotations, residual
  // vector and control words on the device with their pinned host mirror, and
  // the iteration count of the last cycle (the size of the next first batch)
  const int* gate = nullptr;
  const double* vscale = nullptr;   // scale of the stored column a device-driven product reads (VolArgs)
  bool device_gmres = true;
  double* d_gm = nullptr;
  double* h_gm = nullptr;
  int gm_last_k = 4;
  cudaStream_t cap_stream = nullptr;            // private stream the graphs are captured on
  bool jvp_graph_ok = true;
  int* d_jidx = nullptr;
  int* h_jidx = nullptr;                        // pinned, h_jidx[j] = j
  // adaptation workspaces (lazily allocated)
  double* d_xfer = nullptr;              // prolongation / projection matrices [Po][Pn][6][6]
  int* d_adapt_i32 = nullptr;
  int8_t* d_adapt_i8 = nullptr;
  double* d_adapt_f64 = nullptr;
  int64_t* d_old_state_off = nullptr;
  int64_t* d_new_state_off = nullptr;
  int32_t* d_old_elem_slot = nullptr;
  int8_t* d_old_slot_p = nullptr;
  int* h_flag = nullptr;
};

namespace frgb {
void clear_work_cache(fr_ctx* c);
fr_status rebuild_work_table(fr_ctx* c);
void clear_graphs(fr_ctx* c);
void collect_graph_timers(fr_ctx* c);
// launchers (kernels_*.cu)
fr_status launch_residual(fr_ctx* c, const void* q, void* R, fr_prec prec, cudaStream_t s);
fr_status launch_jvp_exact(fr_ctx* c, const void* q, const void* v, void* Jv, fr_prec prec,
                           cudaStream_t s);
fr_status launch_vjp(fr_ctx* c, const void* q, const void* w, void* JTw, fr_prec prec,
                     cudaStream_t s);
fr_status launch_pack(fr_ctx* c, const double* canon, void* q, fr_prec prec, bool unpack,
                      cudaStream_t s);
void set_error(const std::string& msg);
fr_status cuda_check(cudaError_t e, const char* what);
}  // namespace frgb
