// Internal data structures of libsbfwi (not part of the C ABI).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sbfwi.h"

namespace sbfwi {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SBFWI_CUDA(call)                                   \
  do {                                                     \
    cudaError_t err__ = (call);                            \
    if (err__ != cudaSuccess) return cuda_fail(err__, #call); \
  } while (0)

// RAII device buffer
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e == cudaSuccess) bytes = nbytes;
    else p = nullptr;
    return e;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// One cached device allocation for the forward-field store (hundreds of GB at the
// bench size): freeing and re-allocating it every evaluation costs ~0.2 s, so a
// destroyed forward state hands its store to the cache and the next forward state
// of a similar size on the same device takes it over.  sbfwi_release_cache() frees it.
cudaError_t store_alloc(DevBuf& b, size_t bytes);
void store_release(DevBuf& b);
void store_cache_clear();

// ---------------------------------------------------------------------------
// elimination tree of the global boundary system (nested dissection by
// recursive coordinate bisection of the elements)
// ---------------------------------------------------------------------------
struct TreeNodeDev {
  int32_t s, b;            // separator size (eliminated here), boundary size (passed up)
  int32_t child0, child1;  // -1 for leaves
  int32_t elem;            // leaf: its element; -1 otherwise
  int32_t pad;
  int64_t sep_off;         // into sep_nodes (s ids) and ysep rows
  int64_t bnd_off;         // into bnd_nodes (b ids) and ybnd rows
  int64_t map_off;         // into map0/map1 (s+b entries)
  int64_t X_off;           // factor storage: X (s*s) then G (s*b) then C (b*s)
  int64_t F_off;           // set-up workspace: front (f*f)
  int64_t U_off;           // set-up workspace: update matrix (b*b)
};

struct Task {               // a row range of one tree node, with the node's fields inline
  int32_t node;
  int32_t r0, r1;
  int32_t ksplit;           // lanes that share one output's dot product (1, 2, 4 or 8)
  int32_t s, b;             // separator and boundary sizes of the node
  int32_t leaf;             // 1 if the node is an element (front values come from f_hat)
  int32_t pad;              // the node's height (the dataflow trace's phase)
  int64_t sep_off, bnd_off, map_off, X_off;
};

struct Tree {
  std::vector<TreeNodeDev> nodes;      // post-order; root last
  std::vector<int32_t> level_of;       // height: leaves 0
  int levels = 0;
  std::vector<int32_t> sep_nodes, bnd_nodes;
  std::vector<int32_t> map0, map1;     // per front position: child0 / child1 bnd index, -1 if absent;
                                       // leaves: map0 = local dof of the element
  std::vector<int32_t> src0, src1;     // the same for the solve: >= 0 a row of ybnd (a child's
                                       // boundary); <= -2 the f_hat row -2 - src (element * n_b +
                                       // local dof) of the leaf's own element or of a child leaf
                                       // that eliminates nothing (no solve task); -1 absent
  std::vector<std::vector<int32_t>> nodes_at_level;
  int64_t X_total = 0, F_total = 0, U_total = 0, sep_rows = 0, bnd_rows = 0;
  std::vector<int32_t> sep_owner;      // per global node: tree node that eliminates it
};

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
// Device copies of everything that depends on the mesh only (not on the density
// model), made by the first sbfwi_set_model on a mesh and reused by later ones.
struct MeshDevice {
  int device = -1;
  DevBuf xy, ctr, lines, lloc, dofs, xih, xil, tab;
  DevBuf tree_nodes, sep_nodes, bnd_nodes, map0, map1, src0, src1, level_nodes;
  std::vector<int64_t> level_start;
  DevBuf F, U;                       // factorisation workspaces
  DevBuf fgemm;                      // front product tiles {node, kind, r0, c0} (front_gemm_kernel)
  std::vector<int64_t> fgemm_start;  // per level: first G/C tile, first U tile, end
  std::vector<int8_t> fgemm_level;   // per level: products by tiles (1) or in front_factor_kernel (0)
  // bilinear map of one fine grid: base cell and clamping of every nodal point, and
  // the transpose as CSR grid cell -> (point*4 + corner) sorted by point
  // (3-D meshes: trilinear, point*8 + corner)
  bool grid_ready = false;
  int64_t gx = 0, gy = 0, gz = 1;
  double lx = 0, ly = 0, lz = 0;
  DevBuf cell, clamp, cell_ptr, cell_list;
  DevBuf nbe, lptr, api_map;         // n_b per element, first line per element, Mesh::api_to_lib
  // nodal gradient operator (CSR, rows 2q and 2q+1: x and y components at nodal point q)
  bool grad_ready = false;
  DevBuf grad_ptr, grad_col, grad_val;
  // elements at each global node (CSR node -> e * nb + local dof), for the exact adjoint
  bool inc_ready = false;
  DevBuf inc_ptr, inc_list;
};

constexpr int kMaxBoundaryNodes = 40;   // largest n_b of an element

// Elements may have different numbers of boundary nodes n_b(e).  Every per-element array
// is laid out with the largest count, nb, as its stride: local dofs j >= n_b(e) are
// padding, mapped to the extra global node n_nodes, whose state stays zero, and their
// rows and columns of every element operator are zero, so they stay zero through the
// time loop and never reach the global system.
// A 3-D mesh (dim = 3) has the same arrays with surface elements in place of line
// elements: node_xy and centre_xy hold three coordinates per point, line_nodes and
// line_local hold (p+1)^2 nodes per quadrilateral face in tensor order (fpp = nodes per
// boundary element: p+1 in 2-D, (p+1)^2 in 3-D), L counts faces.
struct Mesh {
  int64_t n_elem = 0, n_nodes = 0, n_lines = 0;
  int p = 0, n_r = 0, nb = 0, n = 0, L = 0;   // n = N_r - 1 intervals; nb, L: largest n_b, lines per element
  int dim = 2, fpp = 0;
  double xi0 = 1e-3;
  std::vector<double> node_xy, centre_xy;
  std::vector<int64_t> elem_ptr, line_nodes;
  std::vector<int32_t> nbe;         // [n_elem] n_b of each element
  std::vector<int32_t> dofs;        // [n_elem][nb] global node of each local dof (n_nodes for padding)
  std::vector<int32_t> line_local;  // [n_lines][fpp] local dof of each line (face) position
  bool uneven = false;              // some element has fewer than nb boundary nodes
  Tree tree;
  // nodal points in the library's layout: interior (e, i, j) at (e n + i) nb + j for
  // j < nb (padding included), then the global nodes
  int64_t n_int = 0, n_nodal = 0;
  // nodal points in the caller's layout: interior points of every element without
  // padding (n n_b(e) per element), then the global nodes; api_to_lib maps them
  int64_t n_int_api = 0, n_nodal_api = 0;
  std::vector<int64_t> api_to_lib;  // [n_nodal_api] (empty when !uneven: the layouts agree)
  mutable std::unique_ptr<MeshDevice> dev;   // set-up cache (set_model calls on one mesh must not overlap)
};

int build_tree(Mesh& m);
int ensure_gradient_operator(const Mesh& m, cudaStream_t st);   // MeshDevice::grad_* (setup.cu)
int lfe_element(const double* E0, const double* E1, const double* E2, const double* M0, int nb, double* K,
                double* M);                                        // lfe.cpp

// ---------------------------------------------------------------------------
// model (device resident)
// ---------------------------------------------------------------------------
// Per level and direction the tasks are [block tasks | warp tasks]: a block task is a
// row range of a large front done by the whole block; a warp task is a whole small
// front done by one warp, and `group` warp tasks form one block item.
struct LevelTasks {
  std::vector<int32_t> fwd_start, bwd_start;   // per level: first task index (levels+1 entries)
  std::vector<int32_t> fwd_wstart, bwd_wstart; // per level: first warp task
  std::vector<int32_t> fwd_group, bwd_group;   // per level: warp tasks per block item
  DevBuf fwd, bwd;                              // Task arrays
  DevBuf fwd_meta, bwd_meta;                    // device: start[L+1] | wstart[L] | group[L]
  int shots = 0;                                // tasks were built for this many shots
  int grid = 0;                                 // and this many blocks
  int max_level_items = 0;
  size_t block_doubles = 0;                     // largest staging area of a block task
  // the same tasks as one dataflow: items {first task, count, block?, direction} in
  // topological order, and per tree node [forward tasks | backward tasks | child0 |
  // child1 | nearest ancestor with backward tasks]
  DevBuf flow_items, node_info;
  int n_items = 0, nodes = 0;
  // the dataflow in up to three launches: items [seg[0], seg[1]) are the lower forward
  // levels, [seg[1], seg[2]) the upper levels of both passes, [seg[2], seg[3]) the lower
  // backward levels; the lower levels' tasks fit small_doubles of staging (one launch when
  // every level does: seg[1] == seg[3])
  int flow_seg[4] = {0, 0, 0, 0};
  size_t small_doubles = 0;
  int items(bool fwd, int l) const {
    const auto& st = fwd ? fwd_start : bwd_start;
    const auto& ws = fwd ? fwd_wstart : bwd_wstart;
    const auto& gr = fwd ? fwd_group : bwd_group;
    return (ws[l] - st[l]) + (st[l + 1] - ws[l] + gr[l] - 1) / gr[l];
  }
};

struct Model {
  const Mesh* mesh = nullptr;
  int nb = 0, n = 0;
  int64_t E = 0, N = 0;
  double c = 1, dt = 0, beta = 0.25, gamma = 0.5;
  double a0 = 0, a1 = 0, a2 = 0, c1 = 0, c2 = 0;  // Newmark constants
  int rho_kind = SBFWI_RHO_GRID;
  int64_t gx = 0, gy = 0, gz = 1;
  double lx = 1, ly = 1, lz = 1;
  // element operators, FP64: per element and radial point i = 0..n-1: P_i, Q_i, H_i; then R, T
  DevBuf mats;      // [E][n][3][nb][nb]
  DevBuf rt;        // [E][2][nb][nb]
  DevBuf S;         // [E][nb][nb]  dynamic stiffness
  DevBuf rho_nodal; // [n_nodal] FP64 (hi part of the set-up value)
  // global factors along the elimination tree, followed by copies of the solve's index
  // arrays (src0, src1, sep_nodes, bnd_nodes): one range that the per-step solve
  // keeps resident in L2
  DevBuf factors;
  const int32_t* solve_src0 = nullptr;
  const int32_t* solve_src1 = nullptr;
  const int32_t* solve_sep = nullptr;
  const int32_t* solve_bnd = nullptr;
  size_t solve_bytes = 0;
  DevBuf pts_hi, pts_lo; // [n_nodal][dim] dd location of every nodal point
  // the same operators split into FP16 digits for the tensor-core element kernel
  DevBuf tc_frag, tc_frag_rt, tc_exps, tc_exps_rt;
  bool tc_ready = false;
  bool tc_one_tile = false;   // tc_frag holds one-tile digits although nb > 16 (mixed element kernels)
  DevBuf rho_lo;           // [n_nodal] low part of the set-up's double-double density (re-runs of the set-up)
  // exact discrete adjoint (sbfwi_set_gradient_mode(EXACT)): operators the set-up emits on request
  int grad_mode = SBFWI_GRAD_KERNEL;
  bool exact_ready = false;
  DevBuf xops;             // [E][n][nb][nb] G_i = (modified phi_i)^{-1}
  DevBuf xel;              // [E][6][nb][nb] rho_0, W, Gamma, Y_theta, Y_phi, Y_M
  DevBuf kq;               // [E][L][ng][4] quadrature factors of the coefficient matrices
  DevBuf factors_t;        // the global factors of the transposed matrix (X^T, C^T, G^T per tree node)
  bool lfe = false;        // the comparison method (low-frequency expansion, sbfwi_set_model_lfe)
  DevBuf lfe_M;            // its element masses [E][nb][nb]; S holds K + a0 M
  int kernel_terms = SBFWI_TERMS_VELOCITY;  // sbfwi_set_kernel_terms
  int elem_pref = SBFWI_ELEMENT_AUTO;     // sbfwi_set_schedule
  int solve_pref = SBFWI_SOLVE_AUTO;
  LevelTasks tasks;        // built for tasks.shots
  const MeshDevice& dev() const { return *mesh->dev; }
};

int build_level_tasks(const Model& md, LevelTasks& lt, int shots, int grid);
int prepare_exact(Model& md, cudaStream_t st);   // setup.cu: Model::xops, xel, kq, factors_t
// lfe_setup.cu: the comparison method's K + a0 M and M of every element from E0..M0 [E][4][nb][nb]
int lfe_setup_device(Model& md, const double* Emat, double* S, double* M, cudaStream_t st);

// ---------------------------------------------------------------------------
// exact discrete adjoint kernels (exact.cu)
// ---------------------------------------------------------------------------
struct ExactElemArgs {
  int nb, n, B, epc;
  int64_t E, N;
  double a0, a1, a2;                       // Newmark predictor coefficients
  double cu, cud, cudd, du, dud, dudd;     // u' and u'' of the Newmark update: c_u (u_new - u) + c_ud u' + c_udd u''
  const double* mats;                      // [E][n][3][nb][nb] P, Q, H
  const double* rt;                        // [E][2][nb][nb] R, T
  const double* xops;                      // [E][n][nb][nb] G_i
  const double* xel;                       // [E][6][nb][nb] rho_0, W, Gamma, Y_theta, Y_phi, Y_M
  const int32_t* dofs;                     // [E][nb]
  double* ua; double* uda; double* udda;   // adjoints of the interior u, u', u'' [E][n][nb][B]
  double* s;                               // [E][n][nb][B] up-sweep values
  const double* fbar;                      // [N][B] transposed solve (mu of the flux rows)
  double* mu;                              // [E][n+2][nb][B] mu of rows -1..n
  double* vbn;                             // [E][nb][B] T^T mu_{n+1}
  double* fhat;                            // [E][nb][B] -H_{n-1}^T s_{n-1}
  const double* fu_int;                    // forward u after the step: interior [E][n][nb][B]
  const double* fu_b;                      // and boundary [N][B]
  const double* fa_b;                      // forward u'' after the step, boundary [N][B]
  double* ghost;                           // [E][2][nb][B] u_{-1}, u_{n+1} of the forward solution
  int do_down, do_up;
};

struct ExactBoundaryArgs {
  int64_t N;
  int B;
  double a0, a1, a2, cu, cud, cudd, du, dud, dudd;
  double* ub; double* udb; double* uddb;   // adjoints of the boundary u, u', u'' [N][B]
  double* ext;                             // pre: x_bar of the boundary nodes
  const double* vbn;                       // post: per-element v_bar_n
  const int64_t* inc_ptr;
  const int64_t* inc_list;
};

struct ExactGradArgs {
  int64_t E, N;
  int nb, n, B, Bp, L, ng;
  double h;
  const double* xi;                        // [n+1]
  const double* tab;                       // Gauss weights and Lagrange tables (double-double pairs)
  const int64_t* lptr;                     // [E+1]
  const int32_t* line_local;               // [lines][p+1]
  const int32_t* dofs;
  const double* mu;                        // [E][n+2][nb][B]
  const double* fbar;                      // [N][B]
  const double* fu_int; const double* fu_b;   // forward u after the step
  const double* fa_int; const double* fa_b;   // forward u'' after the step
  const double* ghost;                     // [E][2][nb][B]
  double* gacc;                            // [E][n+1][4][L][ng]
};

struct ExactFinalArgs {
  int64_t E;
  int nb, n, pp, ng, L;
  const int64_t* lptr;
  const int32_t* line_local;
  const double* tab;
  const double* kq;                        // [E][L][ng][4]
  const double* gacc;
  double* g_nodal;                         // interior part of the library's nodal layout
  double* g_bnd;                           // [E][nb] boundary station per element
};

size_t exact_element_smem(int nb, int n, int B, int epc);
int exact_element_launch(const ExactElemArgs& a, cudaStream_t st);
int exact_misfit_launch(double* ub, int B, int R, const int64_t* rec, const double* res, int64_t K, int64_t k, double dt,
                        cudaStream_t st);
int exact_boundary_launch(const ExactBoundaryArgs& a, bool post, cudaStream_t st);
int exact_gradient_launch(const ExactGradArgs& a, int p, cudaStream_t st);
int exact_finalize_launch(const ExactFinalArgs& a, const int64_t* inc_ptr, const int64_t* inc_list, int64_t N,
                          double* g_nodal_b, cudaStream_t st);

// tensor-core element operators (tc.cu)
bool tc_supported(int nb, int B);   // the tensor-core kernel is the default for these shapes
bool tc_available(int nb, int B);   // a tensor-core kernel exists for these shapes
int tc_prepare(Model& md, cudaStream_t st);
int tc_prepare_one_tile(Model& md, cudaStream_t st);   // one-tile digits even when n_b is padded beyond 16
int tc_element_launch(const Model& md, int B, int down, int up, double* u, double* ud, double* udd, double* v,
                      const double* ub, const double* udb, const double* uddb, double* q, double* fhat,
                      double* store_int, const double* fwd_int, double* grad_int, double* u_out, cudaStream_t st,
                      const int32_t* elems = nullptr, int64_t n_elems = 0, int* status = nullptr);

struct FwdState {
  Model* model = nullptr;
  int32_t B = 0, R = 0;
  int64_t K = 0;
  std::vector<int64_t> rec;
  int64_t ckpt_every = 0;       // 0: store holds the velocities of every step
  int64_t state_doubles = 0;    // size of one checkpoint
  bool tensor_core_path = false;
  // ckpt_every == 0: [K][n_nodal][B] nodal velocities after every step;
  // ckpt_every == c > 0: [ceil(K/c) - 1][state_doubles] Newmark states before steps c, 2c, ...
  DevBuf store;
  DevBuf store_u;               // full kernel and exact adjoint: [K][n_nodal][B] nodal displacements after every step
  DevBuf store_a;               // exact adjoint: [K][n_nodal][B] nodal accelerations after every step
  bool exact = false;           // written for the exact adjoint (FP64 element kernel, u and u'' kept)
  DevBuf values, nodes;         // wavelets and source nodes, for the recompute (c > 0)
  // the largest store goes to the one-slot cache (the velocities, or the exact adjoint's displacements)
  ~FwdState() {
    if (store.p) store_release(store);
    else store_release(store_u);
  }
};

}  // namespace sbfwi

// opaque handle types of the C ABI
struct sbfwi_mesh : public sbfwi::Mesh {};
struct sbfwi_model : public sbfwi::Model {};
struct sbfwi_fwdstate : public sbfwi::FwdState {};
