// Context creation: validation, metric terms, per-degree buckets and face
// lists; the C-ABI entry points that only need host logic.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "fr_internal.h"

namespace frgb {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

fr_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FR_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FR_ERR_NOMEM : FR_ERR_CUDA;
}

#define FR_TRY(x)                      \
  do {                                 \
    fr_status _st = (x);               \
    if (_st != FR_OK) return _st;      \
  } while (0)
#define FR_CUDA(x) FR_TRY(cuda_check((x), #x))

static int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// ---------------------------------------------------------------------------
// Metric terms of one element at degree p (cross-product form from the
// derivatives of the degree-p interpolant of the element map).
//   vol  [(nd*nd+1)][NSP]   : S[d][j] at k = d*nd + j, |J| at k = nd*nd
//   face [nf][(nd*nd+1)][NFP]: the same extrapolated to every face
// ---------------------------------------------------------------------------
static void element_metrics(const fr_ctx* c, int e, int p, double* vol, double* face) {
  const int nd = c->nd, g = c->geom_order, nn = g + 1, P = p + 1;
  const int NSP = ipow(P, nd), NFP = ipow(P, nd - 1), NK = nd * nd + 1;
  BasisTab<double> B;
  build_basis(p, B);
  double equi[3];
  for (int a = 0; a < nn; ++a) equi[a] = -1.0 + 2.0 * a / g;
  double N1[kPM][3];
  for (int i = 0; i < P; ++i) lagrange_eval(equi, nn, B.x[i], N1[i]);
  const double* X = c->nodes.data() + (size_t)e * ipow(nn, nd) * nd;
  // coordinates at the solution points
  std::vector<double> Xs((size_t)nd * NSP, 0.0);
  for (int sp = 0; sp < NSP; ++sp) {
    int id[3] = {sp % P, (sp / P) % P, nd == 3 ? sp / (P * P) : 0};
    for (int node = 0; node < ipow(nn, nd); ++node) {
      int nid[3] = {node % nn, (node / nn) % nn, nd == 3 ? node / (nn * nn) : 0};
      double w = 1.0;
      for (int d = 0; d < nd; ++d) w *= N1[id[d]][nid[d]];
      for (int cc = 0; cc < nd; ++cc) Xs[cc * NSP + sp] += w * X[node * nd + cc];
    }
  }
  // derivatives dX[d][comp] at the solution points
  std::vector<double> dX((size_t)nd * nd * NSP, 0.0);
  for (int sp = 0; sp < NSP; ++sp) {
    int id[3] = {sp % P, (sp / P) % P, nd == 3 ? sp / (P * P) : 0};
    for (int d = 0; d < nd; ++d) {
      const int stride = ipow(P, d);
      const int base = sp - id[d] * stride;
      for (int cc = 0; cc < nd; ++cc) {
        double acc = 0.0;
        for (int k = 0; k < P; ++k) acc += B.D[id[d]][k] * Xs[cc * NSP + base + k * stride];
        dX[(d * nd + cc) * NSP + sp] = acc;
      }
    }
  }
  for (int sp = 0; sp < NSP; ++sp) {
    auto D = [&](int d, int cc) { return dX[(d * nd + cc) * NSP + sp]; };
    if (nd == 2) {
      vol[0 * NSP + sp] = D(1, 1);    // S[0][0] = y_eta
      vol[1 * NSP + sp] = -D(1, 0);   // S[0][1] = -x_eta
      vol[2 * NSP + sp] = -D(0, 1);   // S[1][0] = -y_xi
      vol[3 * NSP + sp] = D(0, 0);    // S[1][1] = x_xi
      vol[4 * NSP + sp] = D(0, 0) * D(1, 1) - D(1, 0) * D(0, 1);
    } else {
      for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        vol[(i * 3 + 0) * NSP + sp] = D(j, 1) * D(k, 2) - D(j, 2) * D(k, 1);
        vol[(i * 3 + 1) * NSP + sp] = D(j, 2) * D(k, 0) - D(j, 0) * D(k, 2);
        vol[(i * 3 + 2) * NSP + sp] = D(j, 0) * D(k, 1) - D(j, 1) * D(k, 0);
      }
      // det of a[comp][d] = dX[d][comp]
      double a00 = D(0, 0), a01 = D(1, 0), a02 = D(2, 0);
      double a10 = D(0, 1), a11 = D(1, 1), a12 = D(2, 1);
      double a20 = D(0, 2), a21 = D(1, 2), a22 = D(2, 2);
      vol[9 * NSP + sp] = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
                          a02 * (a10 * a21 - a11 * a20);
    }
  }
  // extrapolate every component to every face
  for (int f = 0; f < 2 * nd; ++f) {
    const int d = f / 2, s = f % 2, stride = ipow(P, d);
    for (int t = 0; t < NFP; ++t) {
      int ta = t % P, tb = t / P;
      int id[3];
      if (nd == 2) {
        id[d == 0 ? 1 : 0] = ta;
      } else {
        int ax[2] = {d == 0 ? 1 : 0, d == 2 ? 1 : 2};
        id[ax[0]] = ta;
        id[ax[1]] = tb;
      }
      id[d] = 0;
      if (nd == 2) id[2] = 0;
      int base = id[0] + P * id[1] + (nd == 3 ? P * P * id[2] : 0);
      for (int kk = 0; kk < NK; ++kk) {
        double acc = 0.0;
        for (int k = 0; k < P; ++k) acc += B.ext[s][k] * vol[kk * NSP + base + k * stride];
        face[((size_t)f * NK + kk) * NFP + t] = acc;
      }
    }
  }
}

static bool element_is_affine(const fr_ctx* c, int e) {
  if (c->geom_order != 1) return false;
  const int nd = c->nd;
  const double* X = c->nodes.data() + (size_t)e * ipow(2, nd) * nd;
  auto node = [&](int i, int j, int k, int cc) { return X[(i + 2 * j + 4 * k) * nd + cc]; };
  double scale = 0.0, twist = 0.0;
  for (int cc = 0; cc < nd; ++cc) {
    scale = std::max(scale, std::fabs(node(1, 0, 0, cc) - node(0, 0, 0, cc)));
    scale = std::max(scale, std::fabs(node(0, 1, 0, cc) - node(0, 0, 0, cc)));
    if (nd == 2) {
      twist = std::max(twist, std::fabs(node(0, 0, 0, cc) - node(1, 0, 0, cc) - node(0, 1, 0, cc) +
                                        node(1, 1, 0, cc)));
    } else {
      scale = std::max(scale, std::fabs(node(0, 0, 1, cc) - node(0, 0, 0, cc)));
      // coefficients of xi*eta, xi*zeta, eta*zeta, xi*eta*zeta of the trilinear map
      double t1 = node(0, 0, 0, cc) - node(1, 0, 0, cc) - node(0, 1, 0, cc) + node(1, 1, 0, cc);
      double t2 = node(0, 0, 0, cc) - node(1, 0, 0, cc) - node(0, 0, 1, cc) + node(1, 0, 1, cc);
      double t3 = node(0, 0, 0, cc) - node(0, 1, 0, cc) - node(0, 0, 1, cc) + node(0, 1, 1, cc);
      double t4 = -node(0, 0, 0, cc) + node(1, 0, 0, cc) + node(0, 1, 0, cc) + node(0, 0, 1, cc) -
                  node(1, 1, 0, cc) - node(1, 0, 1, cc) - node(0, 1, 1, cc) + node(1, 1, 1, cc);
      twist = std::max({twist, std::fabs(t1), std::fabs(t2), std::fabs(t3), std::fabs(t4)});
    }
  }
  return twist <= 1e-13 * scale;
}

// ---------------------------------------------------------------------------
// Layout: buckets in ascending (p, id) order, offsets, face lists.
// ---------------------------------------------------------------------------
void collect_graph_timers(fr_ctx* c) {
  for (int k = 0; k < 2; ++k)
    if (c->graph_timers_live[k]) {
      c->timing.accumulate(c->graph_timers[k]);
      c->graph_timers_live[k] = false;
    }
}

void clear_graphs(fr_ctx* c) {
  collect_graph_timers(c);
  for (int k = 0; k < 2; ++k) {
    if (c->jvp_graph[k]) cudaGraphExecDestroy(c->jvp_graph[k]);
    c->jvp_graph[k] = nullptr;
    for (auto& r : c->graph_timers[k]) c->timing.give_back(r);
    c->graph_timers[k].clear();
    c->graph_timers_live[k] = false;
    for (auto& p : c->jvp_graph_key[k]) p = nullptr;
  }
}

// Work table of the multi-bucket launch: tiles of epb_multi elements, ordered
// by decreasing element weight per tile (higher degrees first), bucket order
// kept among equal weights.  Built on the host and uploaded synchronously.
fr_status rebuild_work_table(fr_ctx* c) {
  cudaFree(c->d_work);
  c->d_work = nullptr;
  c->n_work = 0;
  std::vector<std::pair<double, WorkItem>> items;
  for (size_t bi = 0; bi < c->buckets.size(); ++bi) {
    const Bucket& b = c->buckets[bi];
    const int P = b.p + 1, e = epb_multi(c->nd, P);
    for (int f = 0; f < b.count; f += e) {
      const int ne = std::min(e, b.count - f);
      items.push_back({ne * element_weight(c->epb_tab[0][0][1], ipow(P, c->nd), P), WorkItem{(int32_t)bi, (int32_t)f}});
    }
  }
  if (items.empty()) return FR_OK;
  std::stable_sort(items.begin(), items.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<WorkItem> h(items.size());
  for (size_t i = 0; i < items.size(); ++i) h[i] = items[i].second;
  void* d = nullptr;
  if (cudaMalloc(&d, sizeof(WorkItem) * h.size()) != cudaSuccess) {
    cudaGetLastError();  // out of memory: launches go per bucket instead
    return FR_ERR_NOMEM;
  }
  if (cudaMemcpy(d, h.data(), sizeof(WorkItem) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return cuda_check(cudaGetLastError(), "work table upload");
  }
  c->d_work = static_cast<WorkItem*>(d);
  c->n_work = (int)h.size();
  return FR_OK;
}

void clear_work_cache(fr_ctx* c) {
  c->pc_ready = false;   // the layout or the tuning changed: blocks must be rebuilt
  clear_graphs(c);
  rebuild_work_table(c);
}

// The fused JVP's tables: compact-trace bases of the buckets and, when every
// face is interior and conforming, the neighbour of every element face with
// the master / slave assignment of the face records (higher degree, then lower
// element id, then lower face index).
static fr_status build_fused_table(fr_ctx* c, const std::vector<int32_t>& elem_slot) {
  const int nd = c->nd, nf = c->nf, E = c->E;
  const int ct = c->visc ? 2 * c->nv : c->nv;
  int64_t cb = 0;
  std::vector<int> bucket_of_p(kMaxDeg + 1, -1);
  for (size_t k = 0; k < c->buckets.size(); ++k) {
    Bucket& b = c->buckets[k];
    b.ctrace_base = cb;
    cb += (int64_t)b.count * nf * ct * ipow(b.p + 1, nd - 1);
    bucket_of_p[b.p] = (int)k;
  }
  c->fused_ok = c->bgroups.empty() && cb <= c->trace_cap;
  // the compact face kernel finds a block at the trace-gradient offset scaled
  // by ct / nvt: true when every bucket's compact base is its trace base so scaled
  for (const auto& b : c->buckets)
    if (b.trace_base % c->nvt != 0 || b.trace_base / c->nvt * ct != b.ctrace_base) c->fused_ok = false;
  for (const auto& g : c->fgroups)
    if (g.pm != g.ps) c->fused_ok = false;
  if (!c->fused_ok) return FR_OK;
  std::vector<FusedNbr> h((size_t)E * nf);
  for (int s = 0; s < E; ++s) {
    const int e = c->slot_elem[s];
    for (int f = 0; f < nf; ++f) {
      const int n = c->nbr[(size_t)e * nf + f];
      const int g = c->nbr_face[(size_t)e * nf + f];
      if (n < 0 || c->p[n] != c->p[e]) {
        c->fused_ok = false;
        return FR_OK;
      }
      const bool master = e < n || (e == n && f < g);
      const Bucket& b = c->buckets[bucket_of_p[c->p[n]]];
      FusedNbr r;
      r.nloc = elem_slot[n] - b.slot_begin;
      r.nelem = n;
      r.g = g;
      r.code = (int32_t)(uint8_t)c->orient[(size_t)e * nf + f] | (master ? 256 : 0);
      h[(size_t)s * nf + f] = r;
    }
  }
  if (!c->d_fnbr) FR_CUDA(cudaMalloc(&c->d_fnbr, sizeof(FusedNbr) * (size_t)E * nf));
  FR_CUDA(cudaMemcpy(c->d_fnbr, h.data(), sizeof(FusedNbr) * h.size(), cudaMemcpyHostToDevice));
  return FR_OK;
}

fr_status build_layout(fr_ctx* c) {
  const int nd = c->nd, nv = c->nv, nf = c->nf, E = c->E;
  c->pc_ready = false;
  clear_graphs(c);
  // free previous face groups
  for (auto& g : c->fgroups) cudaFree(g.d_recs);
  for (auto& g : c->bgroups) cudaFree(g.d_recs);
  c->fgroups.clear();
  c->bgroups.clear();
  c->buckets.clear();
  c->slot_elem.resize(E);
  std::vector<int32_t> elem_slot(E);
  int slot = 0;
  int64_t sbase = 0, tbase = 0, obase = 0;
  for (int p = c->p_min; p <= c->p_max; ++p) {
    Bucket b;
    b.p = p;
    b.slot_begin = slot;
    b.state_base = sbase;
    b.trace_base = tbase;
    b.out_base = obase;
    for (int e = 0; e < E; ++e)
      if (c->p[e] == p) {
        elem_slot[e] = slot;
        c->slot_elem[slot++] = e;
      }
    b.count = slot - b.slot_begin;
    const int P = p + 1, NSP = ipow(P, nd), NFP = ipow(P, nd - 1);
    sbase += (int64_t)b.count * nv * NSP;
    tbase += (int64_t)b.count * nf * c->nvt * NFP;
    obase += (int64_t)b.count * nf * 3 * nv * NFP;
    if (b.count > 0) c->buckets.push_back(b);
  }
  c->n_dof = sbase;
  // per-slot host tables
  std::vector<int64_t> canon_off(E + 1, 0), state_off(E), trace_off(E), out_off(E);
  for (int e = 0; e < E; ++e) canon_off[e + 1] = canon_off[e] + (int64_t)nv * ipow(c->p[e] + 1, nd);
  std::vector<int64_t> slot_canon(E);
  std::vector<int8_t> slot_p(E);
  for (const auto& b : c->buckets) {
    const int P = b.p + 1, NSP = ipow(P, nd), NFP = ipow(P, nd - 1);
    for (int i = 0; i < b.count; ++i) {
      const int s = b.slot_begin + i, e = c->slot_elem[s];
      state_off[e] = b.state_base + (int64_t)i * nv * NSP;
      trace_off[e] = b.trace_base + (int64_t)i * nf * c->nvt * NFP;
      out_off[e] = b.out_base + (int64_t)i * nf * 3 * nv * NFP;
      slot_canon[s] = canon_off[e];
      slot_p[s] = (int8_t)b.p;
    }
  }
  std::vector<int64_t> slot_state(E);
  for (int s = 0; s < E; ++s) slot_state[s] = state_off[c->slot_elem[s]];
  FR_CUDA(cudaMemcpy(c->d_slot_elem, c->slot_elem.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice));
  FR_CUDA(cudaMemcpy(c->d_elem_slot, elem_slot.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice));
  FR_CUDA(cudaMemcpy(c->d_canon_off, slot_canon.data(), sizeof(int64_t) * E, cudaMemcpyHostToDevice));
  FR_CUDA(cudaMemcpy(c->d_state_off, slot_state.data(), sizeof(int64_t) * E, cudaMemcpyHostToDevice));
  FR_CUDA(cudaMemcpy(c->d_slot_p, slot_p.data(), E, cudaMemcpyHostToDevice));

  // faces: master = higher degree; ties -> lower element id, then lower face
  std::map<std::pair<int, int>, std::vector<FaceRec>> inter;
  std::map<std::pair<int, int>, std::vector<BndRec>> bnd;
  for (int e = 0; e < E; ++e) {
    const int pe = c->p[e];
    const int NFPe = ipow(pe + 1, nd - 1);
    for (int f = 0; f < nf; ++f) {
      const int n = c->nbr[(size_t)e * nf + f];
      const int64_t mt = trace_off[e] + (int64_t)f * c->nvt * NFPe;
      const int64_t mo = out_off[e] + (int64_t)f * 3 * nv * NFPe;
      if (n < 0) {
        bnd[{pe, n}].push_back(BndRec{mt, mo, e, f});
        continue;
      }
      const int g = c->nbr_face[(size_t)e * nf + f];
      const int pn = c->p[n];
      const bool master = pe > pn || (pe == pn && (e < n || (e == n && f < g)));
      if (!master) continue;
      const int NFPn = ipow(pn + 1, nd - 1);
      FaceRec r;
      r.mt = mt;
      r.mo = mo;
      r.st = trace_off[n] + (int64_t)g * c->nvt * NFPn;
      r.so = out_off[n] + (int64_t)g * 3 * nv * NFPn;
      r.me = e;
      r.se = n;
      r.mf = f;
      r.sf = g;
      r.orient = c->orient[(size_t)e * nf + f];
      auto& v = inter[{pe, pn}];
      r.idx = (int32_t)v.size();
      v.push_back(r);
    }
  }
  int64_t sc = 0;
  for (auto& kv : inter) {
    // master-face direction as the major key (element order kept within a
    // direction): warps then see one normal axis, which the diagonal-metric
    // face kernel branches on
    std::stable_sort(kv.second.begin(), kv.second.end(),
                     [](const FaceRec& a, const FaceRec& b) { return (a.mf >> 1) < (b.mf >> 1); });
    FaceGroup g;
    g.pm = kv.first.first;
    g.ps = kv.first.second;
    g.n = (int)kv.second.size();
    if (g.pm != g.ps) {
      g.scratch_base = sc;
      sc += (int64_t)g.n * 4 * nv * ipow(g.pm + 1, nd - 1);
    }
    FR_CUDA(cudaMalloc(&g.d_recs, sizeof(FaceRec) * g.n));
    FR_CUDA(cudaMemcpy(g.d_recs, kv.second.data(), sizeof(FaceRec) * g.n, cudaMemcpyHostToDevice));
    c->fgroups.push_back(g);
  }
  for (auto& kv : bnd) {
    BndGroup g;
    g.p = kv.first.first;
    g.kind = kv.first.second;
    g.n = (int)kv.second.size();
    FR_CUDA(cudaMalloc(&g.d_recs, sizeof(BndRec) * g.n));
    FR_CUDA(cudaMemcpy(g.d_recs, kv.second.data(), sizeof(BndRec) * g.n, cudaMemcpyHostToDevice));
    c->bgroups.push_back(g);
  }
  if (sc > c->scratch_cap) {
    set_error("mortar scratch exceeds its capacity");
    return FR_ERR_INVALID;
  }
  FR_TRY(build_fused_table(c, elem_slot));
  rebuild_work_table(c);   // a failure leaves no table: launches go per bucket
  return FR_OK;
}

template <typename T>
static fr_status upload_cast(const std::vector<double>& h, T** d) {
  std::vector<T> tmp(h.begin(), h.end());
  FR_CUDA(cudaMalloc(d, sizeof(T) * std::max<size_t>(tmp.size(), 1)));
  FR_CUDA(cudaMemcpy(*d, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice));
  return FR_OK;
}

static fr_status create_impl(const fr_mesh_desc* m, const fr_physics* ph, const fr_limits* lim,
                             fr_ctx* c) {
  if (!m || !ph || !lim || !m->nodes || !m->nbr || !m->nbr_face || !m->orient || !m->p) {
    set_error("fr_create: null argument");
    return FR_ERR_INVALID;
  }
  if ((m->nd != 2 && m->nd != 3) || m->n_elem <= 0 || (m->geom_order != 1 && m->geom_order != 2)) {
    set_error("fr_create: nd must be 2 or 3, n_elem > 0, geom_order 1 or 2");
    return FR_ERR_INVALID;
  }
  if (lim->p_min < 1 || lim->p_max > kMaxDeg || lim->p_min > lim->p_max) {
    set_error("fr_create: need 1 <= p_min <= p_max <= 5");
    return FR_ERR_INVALID;
  }
  if (!(ph->gamma > 1.0) || ph->mu < 0.0 || (ph->mu > 0.0 && !(ph->Pr > 0.0)) ||
      (ph->flux != FR_FLUX_RUSANOV && ph->flux != FR_FLUX_ROE)) {
    set_error("fr_create: need gamma > 1, mu >= 0, Pr > 0 and a known common flux");
    return FR_ERR_INVALID;
  }
  c->nd = m->nd;
  c->nv = m->nd + 2;
  c->nf = 2 * m->nd;
  c->E = m->n_elem;
  c->geom_order = m->geom_order;
  c->p_min = lim->p_min;
  c->p_max = lim->p_max;
  c->visc = ph->mu > 0.0;
  c->phys.gamma = ph->gamma;
  c->phys.mu = ph->mu;
  c->phys.Pr = ph->Pr;
  c->phys.kappa = c->visc ? ph->mu * ph->gamma / ((ph->gamma - 1.0) * ph->Pr) : 0.0;
  for (int v = 0; v < 5; ++v) c->phys.q_inf[v] = ph->q_inf[v];
  c->phys.flux = ph->flux;
  const int nd = c->nd, nf = c->nf, E = c->E, nn = c->geom_order + 1;
  c->nodes.assign(m->nodes, m->nodes + (size_t)E * ipow(nn, nd) * nd);
  c->nbr.assign(m->nbr, m->nbr + (size_t)E * nf);
  c->nbr_face.assign(m->nbr_face, m->nbr_face + (size_t)E * nf);
  c->orient.assign(m->orient, m->orient + (size_t)E * nf);
  c->p.assign(m->p, m->p + E);
  for (int e = 0; e < E; ++e) {
    if (c->p[e] < c->p_min || c->p[e] > c->p_max) {
      set_error("fr_create: element degree outside [p_min, p_max]");
      return FR_ERR_INVALID;
    }
    for (int f = 0; f < nf; ++f) {
      const int n = c->nbr[(size_t)e * nf + f];
      if (n >= E || (n < 0 && n != FR_BC_WALL && n != FR_BC_FARFIELD)) {
        set_error("fr_create: bad neighbour index");
        return FR_ERR_INVALID;
      }
      if (n >= 0) {
        const int g = c->nbr_face[(size_t)e * nf + f];
        if (g < 0 || g >= nf || c->nbr[(size_t)n * nf + g] != e || c->nbr_face[(size_t)n * nf + g] != f) {
          set_error("fr_create: face connectivity is not symmetric");
          return FR_ERR_INVALID;
        }
        const int o = c->orient[(size_t)e * nf + f];
        if (o < 0 || o > 7 || (nd == 2 && (o & 5))) {
          set_error("fr_create: bad orientation code");
          return FR_ERR_INVALID;
        }
      }
    }
  }
  FR_CUDA(cudaGetDevice(&c->device));
  c->nvt = c->visc ? (1 + nd) * c->nv : c->nv;

  // basis and mortar tables
  std::vector<BasisTab<double>> b64(kPM + 1);
  std::vector<BasisTab<float>> b32(kPM + 1);
  for (int P = 2; P <= kPM; ++P) {
    build_basis(P - 1, b64[P]);
    const double* src = reinterpret_cast<const double*>(&b64[P]);
    float* dst = reinterpret_cast<float*>(&b32[P]);
    for (size_t k = 0; k < sizeof(BasisTab<double>) / sizeof(double); ++k) dst[k] = (float)src[k];
  }
  std::vector<MortarTab<double>> m64((kPM + 1) * (kPM + 1));
  std::vector<MortarTab<float>> m32((kPM + 1) * (kPM + 1));
  for (int Pm = 2; Pm <= kPM; ++Pm)
    for (int Ps = 2; Ps < Pm; ++Ps) {
      auto& t = m64[Pm * (kPM + 1) + Ps];
      build_mortar(Ps - 1, Pm - 1, t);
      const double* src = reinterpret_cast<const double*>(&t);
      float* dst = reinterpret_cast<float*>(&m32[Pm * (kPM + 1) + Ps]);
      for (size_t k = 0; k < sizeof(MortarTab<double>) / sizeof(double); ++k) dst[k] = (float)src[k];
    }
  // the same tables rounded to bfloat16 (nearest, ties to even), kept in float
  auto bf16 = [](float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
  };
  std::vector<BasisTab<float>> b16(b32);
  std::vector<MortarTab<float>> m16(m32);
  for (auto& t : b16) {
    float* f = reinterpret_cast<float*>(&t);
    for (size_t k = 0; k < sizeof(BasisTab<float>) / sizeof(float); ++k) f[k] = bf16(f[k]);
  }
  for (auto& t : m16) {
    float* f = reinterpret_cast<float*>(&t);
    for (size_t k = 0; k < sizeof(MortarTab<float>) / sizeof(float); ++k) f[k] = bf16(f[k]);
  }
  FR_CUDA(cudaMalloc(&c->d_basis16, sizeof(BasisTab<float>) * b16.size()));
  FR_CUDA(cudaMemcpy(c->d_basis16, b16.data(), sizeof(BasisTab<float>) * b16.size(), cudaMemcpyHostToDevice));
  FR_CUDA(cudaMalloc(&c->d_mortar16, sizeof(MortarTab<float>) * m16.size()));
  FR_CUDA(cudaMemcpy(c->d_mortar16, m16.data(), sizeof(MortarTab<float>) * m16.size(), cudaMemcpyHostToDevice));
  FR_CUDA(cudaMalloc(&c->d_basis64, sizeof(BasisTab<double>) * b64.size()));
  FR_CUDA(cudaMalloc(&c->d_basis32, sizeof(BasisTab<float>) * b32.size()));
  FR_CUDA(cudaMemcpy(c->d_basis64, b64.data(), sizeof(BasisTab<double>) * b64.size(), cudaMemcpyHostToDevice));
  FR_CUDA(cudaMemcpy(c->d_basis32, b32.data(), sizeof(BasisTab<float>) * b32.size(), cudaMemcpyHostToDevice));
  FR_CUDA(cudaMalloc(&c->d_mortar64, sizeof(MortarTab<double>) * m64.size()));
  FR_CUDA(cudaMalloc(&c->d_mortar32, sizeof(MortarTab<float>) * m32.size()));
  FR_CUDA(cudaMemcpy(c->d_mortar64, m64.data(), sizeof(MortarTab<double>) * m64.size(), cudaMemcpyHostToDevice));
  FR_CUDA(cudaMemcpy(c->d_mortar32, m32.data(), sizeof(MortarTab<float>) * m32.size(), cudaMemcpyHostToDevice));

  // geometry
  c->affine = true;
  for (int e = 0; e < E && c->affine; ++e) c->affine = element_is_affine(c, e);
  const int NK = nd * nd + 1, NKV = geo_nk_vol(nd), NKF = geo_nk_face(nd);
  // the derived components of one point: src holds S and |J| with stride `ss`
  auto derive = [nd, NK](const double* src, int64_t ss, double* dst, int64_t ds, bool face_terms) {
    for (int k = 0; k < NK; ++k) dst[k * ds] = src[k * ss];
    dst[NK * ds] = 1.0 / src[(NK - 1) * ss];
    if (!face_terms) return;
    for (int d = 0; d < nd; ++d) {
      double a2 = 0.0;
      for (int j = 0; j < nd; ++j) a2 += src[(d * nd + j) * ss] * src[(d * nd + j) * ss];
      const double a = std::sqrt(a2);
      dst[(NK + 1 + d) * ds] = a;
      dst[(NK + 1 + nd + d) * ds] = 1.0 / a;
    }
  };
  if (c->affine) {
    // one set of constants per element serves both views (vol uses the first NKV)
    std::vector<double> g((size_t)E * NKF);
    bool diag = nd == 3;
    for (int e = 0; e < E; ++e) {
      // constant metrics: evaluate at degree 0 would be degenerate; use p = 1, first point
      std::vector<double> v1((size_t)NK * ipow(2, nd)), f1((size_t)nf * NK * ipow(2, nd - 1));
      element_metrics(c, e, 1, v1.data(), f1.data());
      // axis-aligned box: the off-diagonal metric terms are rounding noise of
      // the metric evaluation; they are set to exact zeros
      double smax = 0.0, offmax = 0.0;
      for (int d = 0; d < nd; ++d)
        for (int j = 0; j < nd; ++j) {
          const double x = std::fabs(v1[(size_t)(d * nd + j) * ipow(2, nd)]);
          smax = std::max(smax, x);
          if (d != j) offmax = std::max(offmax, x);
        }
      if (offmax <= 1e-13 * smax) {
        for (int d = 0; d < nd; ++d)
          for (int j = 0; j < nd; ++j)
            if (d != j) v1[(size_t)(d * nd + j) * ipow(2, nd)] = 0.0;
      } else {
        diag = false;
      }
      derive(v1.data(), ipow(2, nd), g.data() + (size_t)e * NKF, 1, true);
    }
    c->diag_mesh = diag;
    c->diag = c->diag_mesh && c->use_diag;
    FR_TRY(upload_cast(g, &c->d_gaff64));
    FR_TRY(upload_cast(g, &c->d_gaff32));
  } else {
    for (int p = c->p_min; p <= c->p_max; ++p) {
      const int P = p + 1, NSP = ipow(P, nd), NFP = ipow(P, nd - 1);
      std::vector<double> vol((size_t)E * NKV * NSP), face((size_t)E * nf * NKF * NFP);
#pragma omp parallel for schedule(static)
      for (int e = 0; e < E; ++e) {
        std::vector<double> v0((size_t)NK * NSP), f0((size_t)nf * NK * NFP);
        element_metrics(c, e, p, v0.data(), f0.data());
        double* ve = vol.data() + (size_t)e * NKV * NSP;
        double* fe = face.data() + (size_t)e * nf * NKF * NFP;
        for (int sp = 0; sp < NSP; ++sp) derive(v0.data() + sp, NSP, ve + sp, NSP, false);
        for (int f = 0; f < nf; ++f)
          for (int t = 0; t < NFP; ++t)
            derive(f0.data() + (size_t)f * NK * NFP + t, NFP, fe + (size_t)f * NKF * NFP + t, NFP, true);
      }
      FR_TRY(upload_cast(vol, &c->d_gvol64[p]));
      FR_TRY(upload_cast(vol, &c->d_gvol32[p]));
      FR_TRY(upload_cast(face, &c->d_gface64[p]));
      FR_TRY(upload_cast(face, &c->d_gface32[p]));
    }
  }

  // capacities (all elements at p_max)
  {
    const int P = c->p_max + 1, NSP = ipow(P, nd), NFP = ipow(P, nd - 1);
    c->n_dof_cap = (int64_t)E * c->nv * NSP;
    c->trace_cap = (int64_t)E * nf * c->nvt * NFP;
    c->fout_cap = (int64_t)E * nf * 3 * c->nv * NFP;
    c->scratch_cap = (int64_t)E * nf * 4 * c->nv * NFP;   // bound on all mortar groups
  }
  FR_CUDA(cudaMalloc(&c->d_trace_q, sizeof(double) * c->trace_cap));
  FR_CUDA(cudaMalloc(&c->d_trace_v, sizeof(double) * c->trace_cap));
  FR_CUDA(cudaMalloc(&c->d_fout, sizeof(double) * c->fout_cap));
  FR_CUDA(cudaMalloc(&c->d_scratch, sizeof(double) * std::max<int64_t>(c->scratch_cap, 1)));
  FR_CUDA(cudaMalloc(&c->d_slot_elem, sizeof(int32_t) * E));
  FR_CUDA(cudaMalloc(&c->d_elem_slot, sizeof(int32_t) * E));
  FR_CUDA(cudaMalloc(&c->d_canon_off, sizeof(int64_t) * E));
  FR_CUDA(cudaMalloc(&c->d_state_off, sizeof(int64_t) * E));
  FR_CUDA(cudaMalloc(&c->d_slot_p, E));
  FR_CUDA(cudaMalloc(&c->d_nbr, sizeof(int32_t) * E * nf));
  FR_CUDA(cudaMalloc(&c->d_status, sizeof(int)));
  FR_CUDA(cudaMemset(c->d_status, 0, sizeof(int)));
  FR_CUDA(cudaMemcpy(c->d_nbr, c->nbr.data(), sizeof(int32_t) * E * nf, cudaMemcpyHostToDevice));
  return build_layout(c);
}

static void destroy_impl(fr_ctx* c) {
  cudaFree(c->d_basis64);
  cudaFree(c->d_basis32);
  cudaFree(c->d_basis16);
  cudaFree(c->d_mortar16);
  cudaFree(c->d_mortar64);
  cudaFree(c->d_mortar32);
  cudaFree(c->d_gaff64);
  cudaFree(c->d_gaff32);
  for (int p = 0; p <= kMaxDeg; ++p) {
    cudaFree(c->d_gvol64[p]);
    cudaFree(c->d_gvol32[p]);
    cudaFree(c->d_gface64[p]);
    cudaFree(c->d_gface32[p]);
    cudaFree(c->d_gvol_df[p]);
    cudaFree(c->d_gface_df[p]);
  }
  cudaFree(c->d_basis_df);
  cudaFree(c->d_mortar_df);
  cudaFree(c->d_gaff_df);
  cudaFree(c->d_trace_q);
  cudaFree(c->d_trace_v);
  cudaFree(c->d_fout);
  cudaFree(c->d_scratch);
  cudaFree(c->d_fbar);
  cudaFree(c->d_trbar);
  cudaFree(c->d_slot_elem);
  cudaFree(c->d_elem_slot);
  cudaFree(c->d_canon_off);
  cudaFree(c->d_state_off);
  cudaFree(c->d_slot_p);
  cudaFree(c->d_nbr);
  for (auto& g : c->fgroups) cudaFree(g.d_recs);
  for (auto& g : c->bgroups) cudaFree(g.d_recs);
  clear_graphs(c);
  cudaFree(c->d_work);
  c->d_work = nullptr;
  c->n_work = 0;
  cudaFree(c->d_fnbr);
  cudaFree(c->d_status);
  cudaFree(c->d_jidx);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->h_jidx) cudaFreeHost(c->h_jidx);
  cudaFree(c->d_krylov);
  cudaFree(c->d_krylov32);
  cudaFree(c->d_step);
  cudaFree(c->d_pc);
  cudaFree(c->d_pc_off);
  cudaFree(c->d_slot_color);
  cudaFree(c->d_pc_status);
  for (auto& v : c->d_vec64) cudaFree(v);
  for (auto& v : c->d_vec32) cudaFree(v);
  cudaFree(c->d_red);
  if (c->h_red) cudaFreeHost(c->h_red);
  cudaFree(c->d_gm);
  if (c->h_gm) cudaFreeHost(c->h_gm);
  cudaFree(c->d_xfer);
  cudaFree(c->d_adapt_i32);
  cudaFree(c->d_adapt_i8);
  cudaFree(c->d_adapt_f64);
  cudaFree(c->d_old_state_off);
  cudaFree(c->d_new_state_off);
  cudaFree(c->d_old_elem_slot);
  cudaFree(c->d_old_slot_p);
  if (c->h_flag) cudaFreeHost(c->h_flag);
  delete c;
}

}  // namespace frgb

using namespace frgb;

extern "C" {

const char* fr_last_error(void) { return g_last_error.c_str(); }

fr_status fr_create(const fr_mesh_desc* mesh, const fr_physics* phys, const fr_limits* lim,
                    fr_ctx** out) {
  if (!out) {
    set_error("fr_create: out is null");
    return FR_ERR_INVALID;
  }
  *out = nullptr;
  fr_ctx* c = new (std::nothrow) fr_ctx();
  if (!c) return FR_ERR_NOMEM;
  fr_status st = create_impl(mesh, phys, lim, c);
  if (st != FR_OK) {
    destroy_impl(c);
    return st;
  }
  *out = c;
  return FR_OK;
}

fr_status fr_destroy(fr_ctx* ctx) {
  if (!ctx) return FR_ERR_INVALID;
  destroy_impl(ctx);
  return FR_OK;
}

fr_status fr_layout(const fr_ctx* c, fr_layout_info* info) {
  if (!c || !info) return FR_ERR_INVALID;
  std::memset(info, 0, sizeof(*info));
  info->nd = c->nd;
  info->nv = c->nv;
  info->n_elem = c->E;
  info->n_dof = c->n_dof;
  info->n_dof_capacity = c->n_dof_cap;
  info->affine = c->affine ? 1 : 0;
  for (const auto& b : c->buckets) {
    info->bucket_count[b.p] = b.count;
    info->bucket_offset[b.p] = b.state_base;
  }
  return FR_OK;
}

fr_status fr_get_p(const fr_ctx* c, int8_t* p_host) {
  if (!c || !p_host) return FR_ERR_INVALID;
  std::memcpy(p_host, c->p.data(), c->E);
  return FR_OK;
}

}  // extern "C"
