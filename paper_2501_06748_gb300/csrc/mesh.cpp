// Mesh validation, element-local numbering and the elimination tree of the
// global boundary system.
//
// The global system (sum over elements of the dynamic stiffness S_e, Section 3.3:
// "the global algebraic system ... can then be assembled and solved"; the paper
// leaves the solver open) is solved by a multifrontal factorisation ordered by
// nested dissection: elements are split recursively in halves by the median of
// their scaling centres along the longer extent of their bounding box.  A global
// node is eliminated at the smallest subtree that contains every element
// touching it (its separator); what a subtree still shares with the rest of the
// mesh is its boundary and is passed to the parent.  This file builds that tree,
// its separator/boundary lists and the index maps used to assemble fronts and
// right-hand sides; the numerical work runs in CUDA kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>

#include "internal.h"
#include "prof.h"

namespace sbfwi {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SBFWI_ENOMEM : SBFWI_ECUDA;
}

// ---------------------------------------------------------------------------
// elimination tree
// ---------------------------------------------------------------------------
namespace {

struct Builder {
  const Mesh& m;
  std::vector<int32_t> order;           // elements in tree order
  std::vector<int32_t> lo, hi, c0, c1;  // per tree node
  explicit Builder(const Mesh& mm) : m(mm) {}

  int make(int32_t a, int32_t b) {
    int32_t left = -1, right = -1;
    if (b - a > 1) {
      const int D = m.dim;
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int32_t k = a; k < b; ++k)
        for (int d = 0; d < D; ++d) {
          const double x = m.centre_xy[(size_t)D * order[k] + d];
          lo[d] = std::min(lo[d], x);
          hi[d] = std::max(hi[d], x);
        }
      int ax = 0;                        // the longest extent (the first of equal ones)
      for (int d = 1; d < D; ++d)
        if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
      std::stable_sort(order.begin() + a, order.begin() + b, [&](int32_t e1, int32_t e2) {
        for (int k = 0; k < D; ++k) {    // the split axis first, then the others in order
          const int d = k == 0 ? ax : (k <= ax ? k - 1 : k);
          const double p1 = m.centre_xy[(size_t)D * e1 + d], p2 = m.centre_xy[(size_t)D * e2 + d];
          if (p1 != p2) return p1 < p2;
        }
        return e1 < e2;
      });
      int32_t mid = a + (b - a) / 2;
      left = make(a, mid);
      right = make(mid, b);
    }
    lo.push_back(a); hi.push_back(b); c0.push_back(left); c1.push_back(right);
    return (int)lo.size() - 1;
  }
};

}  // namespace

int build_tree(Mesh& m) {
  Tree& t = m.tree;
  t = Tree();
  Builder bd(m);
  bd.order.resize(m.n_elem);
  std::iota(bd.order.begin(), bd.order.end(), 0);
  int root = bd.make(0, (int32_t)m.n_elem);
  const int T = (int)bd.lo.size();
  if (root != T - 1) return fail(SBFWI_EINVAL, "internal: tree root not last");
  std::vector<int32_t> pos_of(m.n_elem);
  for (int32_t k = 0; k < (int32_t)m.n_elem; ++k) pos_of[bd.order[k]] = k;

  // smallest subtree containing all elements of each node
  std::vector<int32_t> pmin(m.n_nodes, INT32_MAX), pmax(m.n_nodes, -1);
  for (int64_t e = 0; e < m.n_elem; ++e)
    for (int j = 0; j < m.nbe[e]; ++j) {
      int32_t g = m.dofs[e * m.nb + j];
      pmin[g] = std::min(pmin[g], pos_of[e]);
      pmax[g] = std::max(pmax[g], pos_of[e]);
    }
  t.sep_owner.assign(m.n_nodes, -1);
  std::vector<std::vector<int32_t>> sep(T), bnd(T);
  for (int64_t g = 0; g < m.n_nodes; ++g) {
    if (pmax[g] < 0) return fail(SBFWI_EINVAL, "node " + std::to_string(g) + " belongs to no element");
    int nd = root;
    while (bd.c0[nd] >= 0) {
      int a = bd.c0[nd], b = bd.c1[nd];
      if (pmax[g] < bd.hi[a]) nd = a;
      else if (pmin[g] >= bd.lo[b]) nd = b;
      else break;
    }
    t.sep_owner[g] = nd;
    sep[nd].push_back((int32_t)g);
  }
  // boundary lists bottom-up (post-order: children before parents)
  for (int nd = 0; nd < T; ++nd) {
    std::vector<int32_t> cand;
    if (bd.c0[nd] < 0) {
      int32_t e = bd.order[bd.lo[nd]];
      for (int j = 0; j < m.nbe[e]; ++j) cand.push_back(m.dofs[(int64_t)e * m.nb + j]);
    } else {
      cand = bnd[bd.c0[nd]];
      cand.insert(cand.end(), bnd[bd.c1[nd]].begin(), bnd[bd.c1[nd]].end());
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int32_t g : cand)
      if (t.sep_owner[g] != nd) bnd[nd].push_back(g);
    std::sort(sep[nd].begin(), sep[nd].end());
  }
  if (!bnd[root].empty()) return fail(SBFWI_EINVAL, "internal: root of elimination tree has a boundary");

  // node records, maps and offsets
  t.nodes.resize(T);
  t.level_of.assign(T, 0);
  int64_t sep_off = 0, bnd_off = 0, map_off = 0, X_off = 0, F_off = 0, U_off = 0;
  for (int nd = 0; nd < T; ++nd) {
    TreeNodeDev& r = t.nodes[nd];
    r.s = (int32_t)sep[nd].size();
    r.b = (int32_t)bnd[nd].size();
    r.child0 = bd.c0[nd];
    r.child1 = bd.c1[nd];
    r.elem = (bd.c0[nd] < 0) ? bd.order[bd.lo[nd]] : -1;
    r.pad = 0;
    r.sep_off = sep_off;
    r.bnd_off = bnd_off;
    r.map_off = map_off;
    r.X_off = X_off;
    r.F_off = F_off;
    r.U_off = U_off;
    const int64_t s = r.s, b = r.b, f = s + b;
    sep_off += s; bnd_off += b; map_off += f;
    X_off += s * s + 2 * s * b;
    F_off += f * f;
    U_off += b * b;
    t.sep_nodes.insert(t.sep_nodes.end(), sep[nd].begin(), sep[nd].end());
    t.bnd_nodes.insert(t.bnd_nodes.end(), bnd[nd].begin(), bnd[nd].end());
    std::vector<int32_t> front = sep[nd];
    front.insert(front.end(), bnd[nd].begin(), bnd[nd].end());
    if (r.elem >= 0) {
      std::map<int32_t, int32_t> local;
      for (int j = 0; j < m.nbe[r.elem]; ++j) local[m.dofs[(int64_t)r.elem * m.nb + j]] = j;
      for (int32_t g : front) {
        const int32_t j = local.at(g);
        t.map0.push_back(j);
        t.map1.push_back(-1);
        t.src0.push_back(-2 - (int32_t)(r.elem * m.nb + j));     // the element's own f_hat row
        t.src1.push_back(-1);
      }
    } else {
      std::map<int32_t, int32_t> in0, in1;
      for (size_t k = 0; k < bnd[r.child0].size(); ++k) in0[bnd[r.child0][k]] = (int32_t)k;
      for (size_t k = 0; k < bnd[r.child1].size(); ++k) in1[bnd[r.child1][k]] = (int32_t)k;
      const int64_t off0 = t.nodes[r.child0].bnd_off, off1 = t.nodes[r.child1].bnd_off;
      // a child leaf that eliminates nothing passes its f_hat through unchanged: the
      // solve reads f_hat directly (encoded -2 - row) and runs no task for it
      auto src_of = [&](int32_t child, int64_t off, int32_t k, int32_t g) -> int32_t {
        const TreeNodeDev& c = t.nodes[child];
        if (c.elem >= 0 && c.s == 0) {
          int32_t j = 0;
          while (m.dofs[(int64_t)c.elem * m.nb + j] != g) ++j;
          return -2 - (int32_t)(c.elem * m.nb + j);
        }
        return (int32_t)(off + k);
      };
      for (int32_t g : front) {
        auto a = in0.find(g), b2 = in1.find(g);
        t.map0.push_back(a == in0.end() ? -1 : a->second);
        t.map1.push_back(b2 == in1.end() ? -1 : b2->second);
        t.src0.push_back(a == in0.end() ? -1 : src_of(r.child0, off0, a->second, g));
        t.src1.push_back(b2 == in1.end() ? -1 : src_of(r.child1, off1, b2->second, g));
      }
      t.level_of[nd] = 1 + std::max(t.level_of[r.child0], t.level_of[r.child1]);
    }
  }
  t.levels = t.level_of[root] + 1;
  t.nodes_at_level.assign(t.levels, {});
  for (int nd = 0; nd < T; ++nd) t.nodes_at_level[t.level_of[nd]].push_back(nd);
  t.X_total = X_off;
  t.F_total = F_off;
  t.U_total = U_off;
  t.sep_rows = sep_off;
  t.bnd_rows = bnd_off;
  if (sep_off != m.n_nodes) return fail(SBFWI_EINVAL, "internal: separators do not cover the nodes");
  return SBFWI_OK;
}

}  // namespace sbfwi

using namespace sbfwi;

namespace sbfwi {

namespace {
std::mutex g_cache_mu;
void* g_cache_p = nullptr;
size_t g_cache_bytes = 0;
int g_cache_device = -1;

void cache_free_locked() {
  if (g_cache_p) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != g_cache_device) cudaSetDevice(g_cache_device);
    cudaFree(g_cache_p);
    if (cur != g_cache_device) cudaSetDevice(cur);
  }
  g_cache_p = nullptr;
  g_cache_bytes = 0;
  g_cache_device = -1;
}
}  // namespace

cudaError_t store_alloc(DevBuf& b, size_t bytes) {
  b.release();
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    // take the cached buffer if it fits without wasting more than a quarter of it
    if (g_cache_p && g_cache_device == dev && g_cache_bytes >= bytes && g_cache_bytes <= bytes + bytes / 3) {
      b.p = g_cache_p;
      b.bytes = g_cache_bytes;
      g_cache_p = nullptr;
      g_cache_bytes = 0;
      g_cache_device = -1;
      return cudaSuccess;
    }
    cache_free_locked();          // the new allocation may need its memory
  }
  return b.alloc(bytes);
}

void store_release(DevBuf& b) {
  if (!b.p) return;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { b.release(); return; }
  std::lock_guard<std::mutex> lock(g_cache_mu);
  cache_free_locked();
  g_cache_p = b.p;
  g_cache_bytes = b.bytes;
  g_cache_device = dev;
  b.p = nullptr;
  b.bytes = 0;
}

void store_cache_clear() {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  cache_free_locked();
}

Profiler& profiler() {
  static Profiler p;
  return p;
}
}  // namespace sbfwi

// the padded dof table, nodal-point layouts and the elimination tree of a validated mesh
static int finish_mesh(Mesh& mm) {
  Mesh* m = &mm;
  const int64_t n_elem = m->n_elem, n_nodes = m->n_nodes;
  const int nb_max = m->nb;
  // padded dof table: padding points at the extra zero node n_nodes
  {
    std::vector<int32_t> padded((size_t)n_elem * nb_max, (int32_t)n_nodes);
    int64_t k = 0;
    for (int64_t e = 0; e < n_elem; ++e)
      for (int j = 0; j < m->nbe[e]; ++j) padded[(size_t)e * nb_max + j] = m->dofs[k++];
    m->dofs.swap(padded);
  }
  m->n_int = m->n_elem * (int64_t)m->n * m->nb;
  m->n_nodal = m->n_int + m->n_nodes;
  m->n_int_api = 0;
  for (int64_t e = 0; e < n_elem; ++e) {
    m->n_int_api += (int64_t)m->n * m->nbe[e];
    if (m->nbe[e] != m->nb) m->uneven = true;
  }
  m->n_nodal_api = m->n_int_api + m->n_nodes;
  if (m->uneven) {
    m->api_to_lib.reserve(m->n_nodal_api);
    for (int64_t e = 0; e < n_elem; ++e)
      for (int i = 0; i < m->n; ++i)
        for (int j = 0; j < m->nbe[e]; ++j) m->api_to_lib.push_back((e * m->n + i) * m->nb + j);
    for (int64_t g = 0; g < n_nodes; ++g) m->api_to_lib.push_back(m->n_int + g);
  }
  return build_tree(*m);
}

extern "C" {

int sbfwi_profile_enable(int on) {
  profiler().on = (on != 0);
  return SBFWI_OK;
}

int sbfwi_profile_read(double* ms, int64_t* intervals, int64_t* launches, int reset) {
  Profiler& p = profiler();
  for (int k = 0; k < kPhases; ++k) {
    if (ms) ms[k] = p.ms[k];
    if (intervals) intervals[k] = p.intervals[k];
    if (launches) launches[k] = p.launches[k];
    if (reset) { p.ms[k] = 0; p.intervals[k] = 0; p.launches[k] = 0; }
  }
  return SBFWI_OK;
}

int sbfwi_profile_solve_levels(double* us, int32_t cap, int32_t* n_slots, int64_t* steps, int reset) {
  Profiler& p = profiler();
  if (n_slots) *n_slots = p.level_acc ? p.level_slots : 0;
  if (steps) *steps = p.level_steps;
  if (!p.level_acc) return SBFWI_OK;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != p.level_device) return fail(SBFWI_ESTATE, "the solve trace was recorded on another device");
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  std::vector<unsigned long long> acc(p.level_slots);
  e = cudaMemcpy(acc.data(), p.level_acc, sizeof(unsigned long long) * p.level_slots, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read solve trace");
  // slots [2L, 4L) hold maxima (not divided by the number of solves)
  const int L2 = p.level_slots / 3;
  if (us)
    for (int k = 0; k < std::min<int>(cap, p.level_slots); ++k) {
      const bool is_max = k >= L2 && k < 2 * L2;
      us[k] = (is_max || !p.level_steps) ? (double)acc[k] / 1e3 : (double)acc[k] / 1e3 / (double)p.level_steps;
    }
  if (reset) {
    e = cudaMemset(p.level_acc, 0, sizeof(unsigned long long) * p.level_slots);
    if (e != cudaSuccess) return cuda_fail(e, "reset solve trace");
    p.level_steps = 0;
  }
  return SBFWI_OK;
}

int sbfwi_profile_solve_flow(double* us, int32_t cap, int32_t* n_slots, int64_t* steps, int reset) {
  Profiler& p = profiler();
  const int phases = p.flow_acc ? (p.flow_stride - 1) / 4 : 0;
  if (n_slots) *n_slots = 4 * phases;
  if (steps) *steps = p.flow_steps;
  if (!p.flow_acc) return SBFWI_OK;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != p.flow_device) return fail(SBFWI_ESTATE, "the solve trace was recorded on another device");
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  const int rows = (int)std::min<int64_t>(p.flow_steps, Profiler::kFlowRows);
  std::vector<unsigned long long> acc((size_t)p.flow_stride * std::max(rows, 1));
  if (rows > 0) {
    e = cudaMemcpy(acc.data(), p.flow_acc, sizeof(unsigned long long) * p.flow_stride * rows, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read solve trace");
  }
  // device phase index: forward level l -> l, backward level l -> L + l; reported in the
  // order the phases run: forward 0..L-1, then backward L-1..0
  const int L = phases / 2;
  std::vector<double> out(4 * (size_t)phases, 0.0);
  for (int q = 0; q < phases; ++q) {
    const int ph = q < L ? q : L + (phases - 1 - q);
    double done = 0, exec = 0, wait = 0, items = 0;
    int solves = 0;
    for (int r = 0; r < rows; ++r) {
      const unsigned long long* row = acc.data() + (size_t)r * p.flow_stride;
      const unsigned long long* f = row + 1 + 4 * ph;
      if (f[3] == 0) continue;
      done += (double)(f[0] - row[0]);
      exec += (double)f[1];
      wait += (double)f[2];
      items += (double)f[3];
      ++solves;
    }
    if (solves == 0) continue;
    out[q] = done / solves / 1e3;
    out[phases + q] = exec / items / 1e3;
    out[2 * phases + q] = wait / items / 1e3;
    out[3 * phases + q] = items / solves;
  }
  if (us)
    for (int k = 0; k < std::min<int>(cap, 4 * phases); ++k) us[k] = out[k];
  if (reset) p.flow_steps = 0;
  return SBFWI_OK;
}

int sbfwi_release_cache(void) {
  store_cache_clear();
  return SBFWI_OK;
}

const char* sbfwi_last_error(void) { return g_last_error.c_str(); }
int sbfwi_version(void) { return 100; }

int sbfwi_build_mesh(sbfwi_mesh** out, const double* node_xy, int64_t n_nodes, const int64_t* elem_ptr,
                     const int64_t* line_nodes, int64_t n_lines, const double* centre_xy, int64_t n_elem,
                     int32_t p, int32_t n_r, double xi0) {
  if (!out) return fail(SBFWI_EINVAL, "out is NULL");
  *out = nullptr;
  if (!node_xy || !elem_ptr || !line_nodes || !centre_xy) return fail(SBFWI_EINVAL, "NULL array");
  if (n_nodes < 1 || n_elem < 1 || n_lines < 1) return fail(SBFWI_EINVAL, "empty mesh");
  if (n_nodes > INT32_MAX / 2 || n_elem > INT32_MAX / 2) return fail(SBFWI_EINVAL, "mesh too large");
  if (p < 1 || p > 8) return fail(SBFWI_EINVAL, "line order p must be in 1..8");
  if (n_r < 3) return fail(SBFWI_EINVAL, "need at least 3 radial points");
  if (!(xi0 > 0.0 && xi0 < 1.0)) return fail(SBFWI_EINVAL, "xi0 must be in (0, 1)");
  if (elem_ptr[0] != 0 || elem_ptr[n_elem] != n_lines) return fail(SBFWI_EINVAL, "elem_ptr must start at 0 and end at n_lines");
  auto m = new sbfwi_mesh();
  m->n_elem = n_elem; m->n_nodes = n_nodes; m->n_lines = n_lines;
  m->p = p; m->n_r = n_r; m->n = n_r - 1; m->xi0 = xi0;
  m->dim = 2; m->fpp = p + 1;
  m->node_xy.assign(node_xy, node_xy + 2 * n_nodes);
  m->centre_xy.assign(centre_xy, centre_xy + 2 * n_elem);
  m->elem_ptr.assign(elem_ptr, elem_ptr + n_elem + 1);
  m->line_nodes.assign(line_nodes, line_nodes + n_lines * (p + 1));
  auto bad = [&](int code, const std::string& msg) { delete m; return fail(code, msg); };
  for (int64_t k = 0; k < n_lines * (p + 1); ++k)
    if (line_nodes[k] < 0 || line_nodes[k] >= n_nodes) return bad(SBFWI_EINVAL, "line node id out of range");
  int nb_max = 0, L_max = 0;
  for (int64_t e = 0; e < n_elem; ++e) {
    const int64_t l0 = elem_ptr[e], l1 = elem_ptr[e + 1];
    const std::string tag = "element " + std::to_string(e) + ": ";
    if (l1 - l0 < 2) return bad(SBFWI_EINVAL, tag + "needs at least two line elements");
    const double x0 = centre_xy[2 * e], y0 = centre_xy[2 * e + 1];
    std::vector<int32_t> order;
    for (int64_t l = l0; l < l1; ++l) {
      const int64_t* ln = line_nodes + l * (p + 1);
      const int64_t* nx = line_nodes + (l + 1 < l1 ? l + 1 : l0) * (p + 1);
      if (ln[p] != nx[0]) return bad(SBFWI_EINVAL, tag + "line elements do not form a closed loop");
      const double xa = node_xy[2 * ln[0]], ya = node_xy[2 * ln[0] + 1];
      const double xb = node_xy[2 * ln[p]], yb = node_xy[2 * ln[p] + 1];
      const double len = std::hypot(xb - xa, yb - ya);
      if (!(len > 0)) return bad(SBFWI_EINVAL, tag + "degenerate line element");
      for (int k = 1; k < p; ++k) {
        const double xe = xa + (xb - xa) * k / p, ye = ya + (yb - ya) * k / p;
        if (std::hypot(node_xy[2 * ln[k]] - xe, node_xy[2 * ln[k] + 1] - ye) > 1e-9 * len)
          return bad(SBFWI_EINVAL, tag + "line nodes must be equally spaced on a straight segment");
      }
      // det J_b = (x_b - x0) y_b,eta - (y_b - y0) x_b,eta; constant along a straight line
      const double det = (xa - x0) * (yb - ya) - (ya - y0) * (xb - xa);
      if (!(det > 1e-14 * len * len)) return bad(SBFWI_EINVAL, tag + "det J_b <= 0 (centre not strictly inside, or lines not counter-clockwise)");
      for (int k = 0; k <= p; ++k)
        if (std::find(order.begin(), order.end(), (int32_t)ln[k]) == order.end()) order.push_back((int32_t)ln[k]);
    }
    const int L = (int)(l1 - l0);
    if ((int)order.size() != L * p) return bad(SBFWI_EINVAL, tag + "boundary nodes repeat along the loop");
    if (L * p > kMaxBoundaryNodes)
      return bad(SBFWI_EUNSUPPORTED, tag + "more than " + std::to_string(kMaxBoundaryNodes) + " boundary nodes");
    nb_max = std::max(nb_max, L * p);
    L_max = std::max(L_max, L);
    m->nbe.push_back(L * p);
    m->dofs.insert(m->dofs.end(), order.begin(), order.end());
    for (int64_t l = l0; l < l1; ++l)
      for (int k = 0; k <= p; ++k) {
        int32_t g = (int32_t)line_nodes[l * (p + 1) + k];
        m->line_local.push_back((int32_t)(std::find(order.begin(), order.end(), g) - order.begin()));
      }
  }
  m->nb = nb_max;
  m->L = L_max;
  int rc = finish_mesh(*m);
  if (rc != SBFWI_OK) { delete m; return rc; }
  *out = m;
  return SBFWI_OK;
}

int sbfwi_build_mesh3d(sbfwi_mesh** out, const double* node_xyz, int64_t n_nodes, const int64_t* elem_ptr,
                       const int64_t* face_nodes, int64_t n_faces, const double* centre_xyz, int64_t n_elem,
                       int32_t p, int32_t n_r, double xi0) {
  if (!out) return fail(SBFWI_EINVAL, "out is NULL");
  *out = nullptr;
  if (!node_xyz || !elem_ptr || !face_nodes || !centre_xyz) return fail(SBFWI_EINVAL, "NULL array");
  if (n_nodes < 1 || n_elem < 1 || n_faces < 1) return fail(SBFWI_EINVAL, "empty mesh");
  if (n_nodes > INT32_MAX / 2 || n_elem > INT32_MAX / 2) return fail(SBFWI_EINVAL, "mesh too large");
  if (p < 1 || p > 4) return fail(SBFWI_EINVAL, "face order p must be in 1..4");
  if (n_r < 3) return fail(SBFWI_EINVAL, "need at least 3 radial points");
  if (!(xi0 > 0.0 && xi0 < 1.0)) return fail(SBFWI_EINVAL, "xi0 must be in (0, 1)");
  if (elem_ptr[0] != 0 || elem_ptr[n_elem] != n_faces) return fail(SBFWI_EINVAL, "elem_ptr must start at 0 and end at n_faces");
  const int pp = p + 1, fpp = pp * pp;
  auto m = new sbfwi_mesh();
  m->n_elem = n_elem; m->n_nodes = n_nodes; m->n_lines = n_faces;
  m->p = p; m->n_r = n_r; m->n = n_r - 1; m->xi0 = xi0;
  m->dim = 3; m->fpp = fpp;
  m->node_xy.assign(node_xyz, node_xyz + 3 * n_nodes);
  m->centre_xy.assign(centre_xyz, centre_xyz + 3 * n_elem);
  m->elem_ptr.assign(elem_ptr, elem_ptr + n_elem + 1);
  m->line_nodes.assign(face_nodes, face_nodes + n_faces * fpp);
  auto bad = [&](int code, const std::string& msg) { delete m; return fail(code, msg); };
  for (int64_t k = 0; k < n_faces * fpp; ++k)
    if (face_nodes[k] < 0 || face_nodes[k] >= n_nodes) return bad(SBFWI_EINVAL, "face node id out of range");
  auto X = [&](int64_t g, int d) { return node_xyz[3 * g + d]; };
  int nb_max = 0, L_max = 0;
  for (int64_t e = 0; e < n_elem; ++e) {
    const int64_t f0 = elem_ptr[e], f1 = elem_ptr[e + 1];
    const std::string tag = "element " + std::to_string(e) + ": ";
    if (f1 - f0 < 4) return bad(SBFWI_EINVAL, tag + "needs at least four faces");
    const double* c = centre_xyz + 3 * e;
    std::vector<int32_t> order;
    std::map<std::pair<int64_t, int64_t>, int> edges;
    for (int64_t f = f0; f < f1; ++f) {
      const int64_t* fn = face_nodes + f * fpp;
      // corners (a, b) = (0,0), (p,0), (p,p), (0,p); the face must be the bilinear patch
      // of its corners with equally spaced nodes
      const int64_t cn[4] = {fn[0], fn[p], fn[p + pp * p], fn[pp * p]};
      double diam = 0;
      for (int k = 0; k < 4; ++k)
        for (int d = 0; d < 3; ++d) diam = std::max(diam, std::fabs(X(cn[k], d) - X(cn[(k + 1) % 4], d)));
      if (!(diam > 0)) return bad(SBFWI_EINVAL, tag + "degenerate face");
      for (int b = 0; b <= p; ++b)
        for (int a = 0; a <= p; ++a) {
          const double u = (double)a / p, v = (double)b / p;
          for (int d = 0; d < 3; ++d) {
            const double want = (1 - u) * (1 - v) * X(cn[0], d) + u * (1 - v) * X(cn[1], d) + u * v * X(cn[2], d) +
                                (1 - u) * v * X(cn[3], d);
            if (std::fabs(X(fn[a + pp * b], d) - want) > 1e-9 * diam)
              return bad(SBFWI_EINVAL, tag + "face nodes must be equally spaced on the bilinear patch of its corners");
          }
        }
      // det J_b = (x_b - x0) . (x_eta x x_zeta) > 0 at the corners and the middle
      for (int k = 0; k < 5; ++k) {
        const double u = k == 4 ? 0.5 : (k == 1 || k == 2 ? 1.0 : 0.0), v = k == 4 ? 0.5 : (k >= 2 ? 1.0 : 0.0);
        double r[3], xe[3], xz[3];
        for (int d = 0; d < 3; ++d) {
          r[d] = (1 - u) * (1 - v) * X(cn[0], d) + u * (1 - v) * X(cn[1], d) + u * v * X(cn[2], d) +
                 (1 - u) * v * X(cn[3], d) - c[d];
          xe[d] = (1 - v) * (X(cn[1], d) - X(cn[0], d)) + v * (X(cn[2], d) - X(cn[3], d));
          xz[d] = (1 - u) * (X(cn[3], d) - X(cn[0], d)) + u * (X(cn[2], d) - X(cn[1], d));
        }
        const double det = r[0] * (xe[1] * xz[2] - xe[2] * xz[1]) + r[1] * (xe[2] * xz[0] - xe[0] * xz[2]) +
                           r[2] * (xe[0] * xz[1] - xe[1] * xz[0]);
        if (!(det > 1e-14 * diam * diam * diam))
          return bad(SBFWI_EINVAL, tag + "det J_b <= 0 (centre not strictly inside, or a face not oriented outward)");
      }
      for (int k = 0; k < 4; ++k) {
        const int64_t u = cn[k], v = cn[(k + 1) % 4];
        edges[{std::min(u, v), std::max(u, v)}] += 1;
      }
      for (int k = 0; k < fpp; ++k)
        if (std::find(order.begin(), order.end(), (int32_t)fn[k]) == order.end()) order.push_back((int32_t)fn[k]);
    }
    for (const auto& ed : edges)
      if (ed.second != 2) return bad(SBFWI_EINVAL, tag + "faces do not close the element (an edge not shared by two faces)");
    const int L = (int)(f1 - f0);
    if ((int)order.size() > kMaxBoundaryNodes)
      return bad(SBFWI_EUNSUPPORTED, tag + "more than " + std::to_string(kMaxBoundaryNodes) + " boundary nodes");
    nb_max = std::max(nb_max, (int)order.size());
    L_max = std::max(L_max, L);
    m->nbe.push_back((int32_t)order.size());
    m->dofs.insert(m->dofs.end(), order.begin(), order.end());
    for (int64_t f = f0; f < f1; ++f)
      for (int k = 0; k < fpp; ++k) {
        const int32_t g = (int32_t)face_nodes[f * fpp + k];
        m->line_local.push_back((int32_t)(std::find(order.begin(), order.end(), g) - order.begin()));
      }
  }
  m->nb = nb_max;
  m->L = L_max;
  int rc = finish_mesh(*m);
  if (rc != SBFWI_OK) { delete m; return rc; }
  *out = m;
  return SBFWI_OK;
}

int sbfwi_mesh_info(const sbfwi_mesh* m, int64_t* info) {
  if (!m || !info) return fail(SBFWI_EINVAL, "NULL argument");
  info[0] = m->n_elem;
  info[1] = m->n_nodes;
  info[2] = m->nb;
  info[3] = m->n_r;
  info[4] = m->n_nodal_api;
  info[5] = m->n_int_api;
  info[6] = m->tree.levels;
  info[7] = m->tree.X_total;
  return SBFWI_OK;
}

void sbfwi_destroy_mesh(sbfwi_mesh* m) { delete m; }

}  // extern "C"
