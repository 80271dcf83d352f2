// Set-up of the path for one density model (per model, not per step).
//
//  1. density on the nodal points (bilinear map of the fine grid, or given);
//  2. per element, one CTA: coefficient matrices E0, E1, E2, M0 at every radial
//     point (Eq. (Es)), radial derivatives of E0 and E1 (central inside,
//     one-sided at xi_0 and xi_n), blocks theta/phi/psi of Eq. (system), and the
//     algorithmic condensation of Section 3.3, all in double-double; the time
//     loop receives, rounded to FP64,
//         P_i = G_i xi_i^2 M0_i,  Q_i = G_i theta_i,  H_i = G_i psi_i   (i = 0..n-1)
//         R = W theta_n - theta_{n+1},  T = W xi_n^2 M0_n,  S = phi_{n+1} - W phi_n
//     with G_i the inverse of the modified pivot block phi_i and W = psi_{n+1} psi_n^{-1};
//  3. multifrontal factorisation of the global boundary matrix sum_e S_e along
//     the elimination tree (FP64, one CTA per front, Gauss-Jordan with partial
//     pivoting inside each separator block).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <memory>
#include <vector>

#include "dd.cuh"
#include "internal.h"
#include "sync.cuh"
#include "prof.h"

namespace sbfwi {

// ---------------------------------------------------------------------------
// host: Gauss-Legendre rule and Lagrange tables in double-double
// ---------------------------------------------------------------------------
namespace {

void legendre_dd(int n, dd x, dd* pn, dd* pnm1) {
  dd p0 = dd_make(1.0), p1 = x;
  if (n == 0) { *pn = p0; *pnm1 = dd_make(0.0); return; }
  for (int k = 2; k <= n; ++k) {
    // p_k = ((2k-1) x p_{k-1} - (k-1) p_{k-2}) / k
    dd t = dd_sub(dd_mul_d(dd_mul(x, p1), 2.0 * k - 1.0), dd_mul_d(p0, k - 1.0));
    dd pk = dd_div(t, dd_make((double)k));
    p0 = p1;
    p1 = pk;
  }
  *pn = p1;
  *pnm1 = p0;
}

// nodes and weights of the ng-point rule, double-double, ascending
void gauss_legendre_dd(int ng, std::vector<dd>& x, std::vector<dd>& w) {
  x.resize(ng);
  w.resize(ng);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < ng; ++k) {
    // Tricomi's estimate of the (k+1)-th largest root, then Newton in double and double-double
    double xd = std::cos(pi * (k + 0.75) / (ng + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = xd;
      for (int j = 2; j <= ng; ++j) { double pj = ((2.0 * j - 1) * xd * p1 - (j - 1.0) * p0) / j; p0 = p1; p1 = pj; }
      if (ng == 1) p0 = 1.0;
      double dp = ng * (xd * p1 - p0) / (xd * xd - 1.0);
      double dx = p1 / dp;
      xd -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    dd xx = dd_make(xd);
    dd pn, pm;
    for (int it = 0; it < 3; ++it) {
      legendre_dd(ng, xx, &pn, &pm);
      dd dp = dd_div(dd_mul_d(dd_sub(dd_mul(xx, pn), pm), (double)ng), dd_sub(dd_mul(xx, xx), dd_make(1.0)));
      xx = dd_sub(xx, dd_div(pn, dp));
    }
    legendre_dd(ng, xx, &pn, &pm);
    dd dp = dd_div(dd_mul_d(dd_sub(dd_mul(xx, pn), pm), (double)ng), dd_sub(dd_mul(xx, xx), dd_make(1.0)));
    dd one_m_x2 = dd_sub(dd_make(1.0), dd_mul(xx, xx));
    w[ng - 1 - k] = dd_div(dd_make(2.0), dd_mul(one_m_x2, dd_mul(dp, dp)));
    x[ng - 1 - k] = xx;
  }
}

// phi_a(eta) and d phi_a / d eta for equally spaced nodes eta_b = -1 + 2b/p
void lagrange_dd(int p, dd eta, dd* phi, dd* dphi) {
  std::vector<dd> nodes(p + 1);
  for (int b = 0; b <= p; ++b) nodes[b] = dd_sub(dd_div(dd_make(2.0 * b), dd_make((double)p)), dd_make(1.0));
  for (int a = 0; a <= p; ++a) {
    dd denom = dd_make(1.0), num = dd_make(1.0), der = dd_make(0.0);
    for (int b = 0; b <= p; ++b) {
      if (b == a) continue;
      denom = dd_mul(denom, dd_sub(nodes[a], nodes[b]));
      num = dd_mul(num, dd_sub(eta, nodes[b]));
    }
    for (int m = 0; m <= p; ++m) {
      if (m == a) continue;
      dd t = dd_make(1.0);
      for (int b = 0; b <= p; ++b)
        if (b != a && b != m) t = dd_mul(t, dd_sub(eta, nodes[b]));
      der = dd_add(der, t);
    }
    phi[a] = dd_div(num, denom);
    dphi[a] = dd_div(der, denom);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_flag(int* status, int code) { atomicCAS(status, 0, code); }

// ---------------------------------------------------------------------------
// 1. density at the nodal points (double-double)
// ---------------------------------------------------------------------------
struct DensityArgs {
  int64_t n_elem, n_nodes, n_int;
  int nb, n;
  const int32_t* nbe;        // n_b of each element: padding points get density 1 at the centre
  const double* node_xy;
  const double* centre_xy;
  const int32_t* dofs;
  const double* xi_hi;
  const double* xi_lo;
  const double* grid;        // [gy][gx] ([gz][gy][gx] in 3-D) or nodal values
  int rho_kind;
  int dim;
  int64_t gx, gy, gz;
  double lx, ly, lz;
  const int32_t* cell_of_point;
  const int8_t* clamp_of_point;
  double* pts_hi;            // [n_nodal][dim]
  double* pts_lo;
  double* rho_hi;            // [n_nodal]
  double* rho_lo;
  int* status;
};

__global__ void density_kernel(DensityArgs a) {
  const int64_t np = a.n_int + a.n_nodes;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
    dd px, py;
    if (q < a.n_int) {
      const int64_t e = q / ((int64_t)a.n * a.nb);
      const int64_t rem = q - e * (int64_t)a.n * a.nb;
      const int i = (int)(rem / a.nb), j = (int)(rem - (int64_t)i * a.nb);
      const double x0 = a.centre_xy[2 * e], y0 = a.centre_xy[2 * e + 1];
      if (j >= a.nbe[e]) {                 // padding: never used by the method
        a.pts_hi[2 * q] = x0; a.pts_lo[2 * q] = 0.0;
        a.pts_hi[2 * q + 1] = y0; a.pts_lo[2 * q + 1] = 0.0;
        a.rho_hi[q] = 1.0; a.rho_lo[q] = 0.0;
        continue;
      }
      const int32_t g = a.dofs[e * a.nb + j];
      const dd xi{a.xi_hi[i], a.xi_lo[i]};
      // x0 + xi (x_j - x0)
      px = dd_add(dd_make(x0), dd_mul(xi, two_sum(a.node_xy[2 * g], -x0)));
      py = dd_add(dd_make(y0), dd_mul(xi, two_sum(a.node_xy[2 * g + 1], -y0)));
    } else {
      const int64_t g = q - a.n_int;
      px = dd_make(a.node_xy[2 * g]);
      py = dd_make(a.node_xy[2 * g + 1]);
    }
    a.pts_hi[2 * q] = px.hi; a.pts_lo[2 * q] = px.lo;
    a.pts_hi[2 * q + 1] = py.hi; a.pts_lo[2 * q + 1] = py.lo;
    dd rho;
    if (a.rho_kind == SBFWI_RHO_NODAL) {
      rho = dd_make(a.grid[q]);
    } else {
      // bilinear interpolation of the cell-centred grid, clamped at the edges
      const int32_t cell = a.cell_of_point[q];
      const int8_t cl = a.clamp_of_point[q];
      const int64_t ix = cell % a.gx, iy = cell / a.gx;
      dd tx, ty;
      if (cl & 1) tx = dd_make(0.0);
      else if (cl & 2) tx = dd_make(1.0);
      else {  // fx = x * gx / lx - 1/2 - ix
        dd fx = dd_div(dd_mul_d(px, (double)a.gx), dd_make(a.lx));
        tx = dd_sub(fx, dd_make(0.5 + (double)ix));
      }
      if (cl & 4) ty = dd_make(0.0);
      else if (cl & 8) ty = dd_make(1.0);
      else {
        dd fy = dd_div(dd_mul_d(py, (double)a.gy), dd_make(a.ly));
        ty = dd_sub(fy, dd_make(0.5 + (double)iy));
      }
      const double* G = a.grid;
      const dd one = dd_make(1.0);
      const dd wx0 = dd_sub(one, tx), wy0 = dd_sub(one, ty);
      dd v = dd_mul(dd_mul(wx0, wy0), dd_make(G[iy * a.gx + ix]));
      v = dd_add(v, dd_mul(dd_mul(tx, wy0), dd_make(G[iy * a.gx + ix + 1])));
      v = dd_add(v, dd_mul(dd_mul(wx0, ty), dd_make(G[(iy + 1) * a.gx + ix])));
      v = dd_add(v, dd_mul(dd_mul(tx, ty), dd_make(G[(iy + 1) * a.gx + ix + 1])));
      rho = v;
    }
    if (!(rho.hi > 0.0)) atomic_flag(a.status, SBFWI_EINVAL);
    a.rho_hi[q] = rho.hi;
    a.rho_lo[q] = rho.lo;
  }
}

// The same for a 3-D mesh: nodal points x0 + xi_i (x_j - x0) in three coordinates and
// trilinear interpolation of the cell-centred [gz][gy][gx] grid, clamped at the edges
__global__ void density3d_kernel(DensityArgs a) {
  const int64_t np = a.n_int + a.n_nodes;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
    dd px[3];
    if (q < a.n_int) {
      const int64_t e = q / ((int64_t)a.n * a.nb);
      const int64_t rem = q - e * (int64_t)a.n * a.nb;
      const int i = (int)(rem / a.nb), j = (int)(rem - (int64_t)i * a.nb);
      const double* c0 = a.centre_xy + 3 * e;
      if (j >= a.nbe[e]) {                 // padding: never used by the method
        for (int d = 0; d < 3; ++d) { a.pts_hi[3 * q + d] = c0[d]; a.pts_lo[3 * q + d] = 0.0; }
        a.rho_hi[q] = 1.0; a.rho_lo[q] = 0.0;
        continue;
      }
      const int32_t g = a.dofs[e * a.nb + j];
      const dd xi{a.xi_hi[i], a.xi_lo[i]};
      for (int d = 0; d < 3; ++d) px[d] = dd_add(dd_make(c0[d]), dd_mul(xi, two_sum(a.node_xy[3 * g + d], -c0[d])));
    } else {
      const int64_t g = q - a.n_int;
      for (int d = 0; d < 3; ++d) px[d] = dd_make(a.node_xy[3 * g + d]);
    }
    for (int d = 0; d < 3; ++d) { a.pts_hi[3 * q + d] = px[d].hi; a.pts_lo[3 * q + d] = px[d].lo; }
    dd rho;
    if (a.rho_kind == SBFWI_RHO_NODAL) {
      rho = dd_make(a.grid[q]);
    } else {
      const int64_t cell = a.cell_of_point[q];
      const int8_t cl = a.clamp_of_point[q];
      const int64_t ix = cell % a.gx, iy = (cell / a.gx) % a.gy, iz = cell / (a.gx * a.gy);
      const int64_t gdim[3] = {a.gx, a.gy, a.gz}, base[3] = {ix, iy, iz};
      const double len[3] = {a.lx, a.ly, a.lz};
      dd t[3];
      for (int d = 0; d < 3; ++d) {
        if (cl & (1 << (2 * d))) t[d] = dd_make(0.0);
        else if (cl & (2 << (2 * d))) t[d] = dd_make(1.0);
        else t[d] = dd_sub(dd_div(dd_mul_d(px[d], (double)gdim[d]), dd_make(len[d])), dd_make(0.5 + (double)base[d]));
      }
      const dd one = dd_make(1.0);
      dd v = dd_make(0.0);
      for (int c = 0; c < 8; ++c) {
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
        const dd w = dd_mul(dd_mul(cx ? t[0] : dd_sub(one, t[0]), cy ? t[1] : dd_sub(one, t[1])),
                            cz ? t[2] : dd_sub(one, t[2]));
        v = dd_add(v, dd_mul(w, dd_make(a.grid[((iz + cz) * a.gy + iy + cy) * a.gx + ix + cx])));
      }
      rho = v;
    }
    if (!(rho.hi > 0.0)) atomic_flag(a.status, SBFWI_EINVAL);
    a.rho_hi[q] = rho.hi;
    a.rho_lo[q] = rho.lo;
  }
}

__global__ void fill_kernel(double* x, int64_t n, double v) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) x[q] = v;
}

// comparison method: every interior nodal point takes the density of its boundary node
// (the density constant along each radial line, Section 3.2)
__global__ void radial_constant_density_kernel(double* rho_hi, double* rho_lo, const int32_t* dofs,
                                               const int32_t* nbe, int64_t n_int, int n, int nb) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_int; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = q / ((int64_t)n * nb);
    const int j = (int)(q % nb);
    if (j >= nbe[e]) continue;
    const int64_t g = n_int + dofs[e * nb + j];
    rho_hi[q] = rho_hi[g];
    rho_lo[q] = rho_lo[g];
  }
}

// lib[map[q]] = api[q]: nodal values from the caller's layout to the padded one
__global__ void scatter_nodal_kernel(const double* api, const int64_t* map, int64_t n, double* lib) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    lib[map[q]] = api[q];
}

// ---------------------------------------------------------------------------
// 2. element set-up (double-double, one CTA per element, one thread per entry)
// ---------------------------------------------------------------------------
struct ElemArgs {
  int nb, n, L, p, ng;        // nb, L: largest n_b and line count (strides of the outputs and smem)
  int dim, fpp, nk;           // 2 or 3; nodes per line (face); geometry factors per Gauss point (4 or 7)
  int64_t e0;                 // first element of this launch
  const int32_t* nbe;         // [E] n_b of each element
  const int64_t* lptr;        // [E+1] first line of each element
  dd* mat_ws;                 // global workspace for the 16 matrices (nullptr: shared memory)
  double* E_out;              // comparison method: E0, E1, E2, M0 of radial point 0 [E][4][nb][nb], then stop
  int64_t n_elem, n_int;
  double c;
  dd mass;                    // 1 / (beta dt^2)
  dd h;                       // radial spacing (1 - xi0) / n
  const double* node_xy;
  const double* centre_xy;
  const int64_t* line_nodes;  // [n_lines][p+1] (elements own consecutive lines)
  const int32_t* line_local;  // [n_lines][p+1]
  const int32_t* dofs;
  const double* rho_hi;
  const double* rho_lo;
  const double* xi_hi;        // [n+1]
  const double* xi_lo;
  const double* tab;          // dd tables (hi,lo pairs): w[ng], phi[ng][fpp], dphi[ng][fpp], (3-D) dphi_zeta[ng][fpp]
                              // (3-D: ng points of the tensor face rule, phi = N, dphi = N_eta)
  double* mats;               // [E][n][3][nb][nb], zero beyond n_b(e)
  double* rt;                 // [E][2][nb][nb]
  double* S;                  // [E][nb][nb]
  // exact discrete adjoint (nullable; see ExactOps in internal.h)
  double* xops;               // [E][n][nb][nb] G_i, the inverse of the modified pivot block phi_i
  double* xel;                // [E][6][nb][nb] rho_0, W, Gamma, Y_theta, Y_phi, Y_M
  double* kq;                 // [E][L][ng][4] quadrature factors of Eq. (Es): c^2 w det (b1.b1),
                              // c^2 w det (b2.b1), c^2 w det (b2.b2), w det
  int* status;
};

struct ElemSmem {
  dd* K;      // [L][ng][nk] geometry factors.  2-D: c^2 w det (b1.b1), c^2 w det (b2.b1),
              // c^2 w det (b2.b2), w det.  3-D: c^2 w det times b1.b1, b2.b1, b3.b1, b2.b2,
              // b2.b3, b3.b3, then w det
  dd* KR;     // [L][ng][nk] the same times rho at the Gauss point
  dd* Eline;  // [L][fpp][fpp][4] per-line (face) contributions
  dd* phi;    // [ng][fpp]
  dd* dphi;   // [ng][fpp]
  dd* dphz;   // [ng][fpp] (3-D)
  dd* mat;    // 16 matrices of n_b(e)^2 (placed nb*nb apart)
  dd* col;    // [nb] Gauss-Jordan factor column
  int* piv;
  int nb, L;  // this element's boundary nodes and lines
  int64_t l0; // its first line
};

__device__ __forceinline__ dd ldd(const double* hi, const double* lo, int64_t k) { return dd{hi[k], lo[k]}; }

// Arithmetic of one radial point of the set-up.  Only the points next to the scaling
// centre need more than binary64: there the first pivot -xi0 E0 / (2h) amplifies
// rounding of the coefficient matrices and blocks by ~1e4.  Points 0..3 (their
// coefficient matrices) and rows 0, 1 (blocks, first elimination, first Thomas step)
// run in double-double; everything farther out in binary64 (the hi part of the dd
// storage, lo = 0), which moves receiver traces by ~1e-13 against an all-extended
// set-up (measured on the CPU with the oracle's extended-precision arithmetic).
struct DDOps {
  static __device__ __forceinline__ dd make(double a) { return dd_make(a); }
  static __device__ __forceinline__ dd add(dd x, dd y) { return dd_add(x, y); }
  static __device__ __forceinline__ dd sub(dd x, dd y) { return dd_sub(x, y); }
  static __device__ __forceinline__ dd mul(dd x, dd y) { return dd_mul(x, y); }
  static __device__ __forceinline__ dd mul_d(dd x, double y) { return dd_mul_d(x, y); }
  static __device__ __forceinline__ dd fma(dd acc, dd x, dd y) { return dd_fma(acc, x, y); }
  static __device__ __forceinline__ dd div(dd x, dd y) { return dd_div(x, y); }
  static __device__ __forceinline__ dd neg(dd x) { return dd_neg(x); }
};
struct F64Ops {
  static __device__ __forceinline__ dd make(double a) { return dd{a, 0.0}; }
  static __device__ __forceinline__ dd add(dd x, dd y) { return dd{x.hi + y.hi, 0.0}; }
  static __device__ __forceinline__ dd sub(dd x, dd y) { return dd{x.hi - y.hi, 0.0}; }
  static __device__ __forceinline__ dd mul(dd x, dd y) { return dd{x.hi * y.hi, 0.0}; }
  static __device__ __forceinline__ dd mul_d(dd x, double y) { return dd{x.hi * y, 0.0}; }
  static __device__ __forceinline__ dd fma(dd acc, dd x, dd y) { return dd{::fma(x.hi, y.hi, acc.hi), 0.0}; }
  static __device__ __forceinline__ dd div(dd x, dd y) { return dd{x.hi / y.hi, 0.0}; }
  static __device__ __forceinline__ dd neg(dd x) { return dd{-x.hi, 0.0}; }
};
constexpr int kExtendedPoints = 4;   // coefficient matrices of points 0..3 in double-double
constexpr int kExtendedRows = 2;     // rows 0, 1 of the condensation in double-double

// E0, E1, E2, M0 of element e at radial point i into the four given matrices
template <class Op>
__device__ void coefficient_matrices(const ElemArgs& a, const ElemSmem& sm, int64_t e, int i,
                                     dd* E0, dd* E1, dd* E2, dd* M0) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nb = sm.nb, L = sm.L, ng = a.ng, pp = a.fpp, nk = a.nk, nbs = a.nb;
  // density at the Gauss points of every line (face), times the geometry factors
  for (int t = tid; t < L * ng; t += nt) {
    const int l = t / ng, g = t - l * ng;
    dd r = Op::make(0.0);
    for (int q = 0; q < pp; ++q) {
      const int j = a.line_local[(sm.l0 + l) * pp + q];
      const int64_t idx = (i < a.n) ? e * (int64_t)a.n * nbs + (int64_t)i * nbs + j : a.n_int + a.dofs[e * nbs + j];
      r = Op::fma(r, sm.phi[g * pp + q], ldd(a.rho_hi, a.rho_lo, idx));
    }
    for (int k = 0; k < nk; ++k) sm.KR[(l * ng + g) * nk + k] = Op::mul(sm.K[(l * ng + g) * nk + k], r);
  }
  __syncthreads();
  // per-line (face) matrices: sum over Gauss points
  for (int t = tid; t < L * pp * pp; t += nt) {
    const int l = t / (pp * pp), ab = t - l * pp * pp, aa = ab / pp, bb = ab - aa * pp;
    dd s0 = Op::make(0.0), s1 = s0, s2 = s0, sm0 = s0;
    for (int g = 0; g < ng; ++g) {
      const dd* kr = sm.KR + (l * ng + g) * nk;
      const dd pa = sm.phi[g * pp + aa], pb = sm.phi[g * pp + bb];
      const dd da = sm.dphi[g * pp + aa], db = sm.dphi[g * pp + bb];
      const dd papb = Op::mul(pa, pb);
      s0 = Op::fma(s0, kr[0], papb);
      if (a.dim == 2) {
        s1 = Op::fma(s1, kr[1], Op::mul(da, pb));
        s2 = Op::fma(s2, kr[2], Op::mul(da, db));
        sm0 = Op::fma(sm0, kr[3], papb);
      } else {
        // B2 = b2 N_eta + b3 N_zeta: E1 += (b2.b1 N_eta,a + b3.b1 N_zeta,a) N_b,
        // E2 += b2.b2 N_eta,a N_eta,b + b2.b3 (N_eta,a N_zeta,b + N_zeta,a N_eta,b) + b3.b3 N_zeta,a N_zeta,b
        const dd za = sm.dphz[g * pp + aa], zb = sm.dphz[g * pp + bb];
        s1 = Op::fma(s1, Op::add(Op::mul(kr[1], da), Op::mul(kr[2], za)), pb);
        dd q2 = Op::mul(kr[3], Op::mul(da, db));
        q2 = Op::fma(q2, kr[4], Op::add(Op::mul(da, zb), Op::mul(za, db)));
        q2 = Op::fma(q2, kr[5], Op::mul(za, zb));
        s2 = Op::add(s2, q2);
        sm0 = Op::fma(sm0, kr[6], papb);
      }
    }
    dd* out = sm.Eline + (size_t)t * 4;
    out[0] = s0; out[1] = s1; out[2] = s2; out[3] = sm0;
  }
  __syncthreads();
  // assemble the element matrices from the lines (faces)
  for (int t = tid; t < nb * nb; t += nt) {
    const int A = t / nb, B = t - A * nb;
    dd s0 = Op::make(0.0), s1 = s0, s2 = s0, s3 = s0;
    for (int l = 0; l < L; ++l) {
      int pa = -1, pb = -1;
      for (int q = 0; q < pp; ++q) {
        const int j = a.line_local[(sm.l0 + l) * pp + q];
        if (j == A) pa = q;
        if (j == B) pb = q;
      }
      if (pa < 0 || pb < 0) continue;
      const dd* v = sm.Eline + ((size_t)(l * pp + pa) * pp + pb) * 4;
      s0 = Op::add(s0, v[0]); s1 = Op::add(s1, v[1]); s2 = Op::add(s2, v[2]); s3 = Op::add(s3, v[3]);
    }
    E0[t] = s0; E1[t] = s1; E2[t] = s2; M0[t] = s3;
  }
  __syncthreads();
}

// Inv = A^{-1} by Gauss-Jordan with partial pivoting; A is destroyed.
template <class Op>
__device__ void gj_inverse(int nb, dd* A, dd* Inv, dd* col, int* piv, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < nb * nb; t += nt) Inv[t] = Op::make((t / nb) == (t % nb) ? 1.0 : 0.0);
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      int best = k;
      double bv = fabs(A[k * nb + k].hi);
      for (int r = k + 1; r < nb; ++r) {
        const double v = fabs(A[r * nb + k].hi);
        if (v > bv) { bv = v; best = r; }
      }
      if (!(bv > 0.0) || !isfinite(bv)) atomic_flag(status, SBFWI_ESINGULAR);
      *piv = best;
    }
    __syncthreads();
    const int pr = *piv;
    if (pr != k) {
      for (int c = tid; c < nb; c += nt) {
        dd t1 = A[k * nb + c]; A[k * nb + c] = A[pr * nb + c]; A[pr * nb + c] = t1;
        dd t2 = Inv[k * nb + c]; Inv[k * nb + c] = Inv[pr * nb + c]; Inv[pr * nb + c] = t2;
      }
    }
    __syncthreads();
    for (int r = tid; r < nb; r += nt) col[r] = A[r * nb + k];
    __syncthreads();
    const dd pinv = Op::div(Op::make(1.0), col[k]);
    for (int t = tid; t < nb * nb; t += nt) {
      const int r = t / nb, c = t - r * nb;
      // row k is only read here; it is normalised after the barrier below
      const dd ak = Op::mul(A[k * nb + c], pinv), ik = Op::mul(Inv[k * nb + c], pinv);
      if (r != k) {
        const dd f = col[r];
        A[t] = Op::sub(A[t], Op::mul(f, ak));
        Inv[t] = Op::sub(Inv[t], Op::mul(f, ik));
      }
    }
    __syncthreads();
    for (int c = tid; c < nb; c += nt) {
      A[k * nb + c] = Op::mul(A[k * nb + c], pinv);
      Inv[k * nb + c] = Op::mul(Inv[k * nb + c], pinv);
    }
    __syncthreads();
  }
}

// C = A * B (all nb x nb, distinct buffers)
template <class Op>
__device__ void mm(int nb, const dd* A, const dd* B, dd* C) {
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int r = t / nb, c = t - r * nb;
    dd s = Op::make(0.0);
    for (int k = 0; k < nb; ++k) s = Op::fma(s, A[r * nb + k], B[k * nb + c]);
    C[t] = s;
  }
  __syncthreads();
}

__global__ void element_setup_kernel(ElemArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t e = a.e0 + blockIdx.x;
  const int ng = a.ng, pp = a.fpp, nk = a.nk, n = a.n, nbs = a.nb;
  const int nb = a.nbe[e], L = (int)(a.lptr[e + 1] - a.lptr[e]);
  const int nn = nb * nb;                 // this element's matrices are dense nb x nb
  const int64_t nns = (int64_t)nbs * nbs; // stride of the padded outputs
  const int tid = threadIdx.x, nt = blockDim.x;
  ElemSmem sm;
  sm.nb = nb; sm.L = L; sm.l0 = a.lptr[e];
  dd* base = reinterpret_cast<dd*>(smem_raw);
  sm.K = base;                     base += a.L * ng * nk;
  sm.KR = base;                    base += a.L * ng * nk;
  sm.Eline = base;                 base += a.L * pp * pp * 4;
  sm.phi = base;                   base += ng * pp;
  sm.dphi = base;                  base += ng * pp;
  sm.dphz = base;                  base += a.dim == 3 ? ng * pp : 0;
  sm.col = base;                   base += nbs;
  if (a.mat_ws) {
    sm.mat = a.mat_ws + (int64_t)blockIdx.x * 16 * nns;
  } else {
    sm.mat = base;                 base += 16 * nns;
  }
  sm.piv = reinterpret_cast<int*>(base);
  const int ms = (int)nns;
  dd* E0w[3] = {sm.mat + 0 * ms, sm.mat + 1 * ms, sm.mat + 2 * ms};
  dd* E1w[3] = {sm.mat + 3 * ms, sm.mat + 4 * ms, sm.mat + 5 * ms};
  dd* E2w[2] = {sm.mat + 6 * ms, sm.mat + 7 * ms};
  dd* M0w[2] = {sm.mat + 8 * ms, sm.mat + 9 * ms};
  dd* th = sm.mat + 10 * ms;
  dd* ph = sm.mat + 11 * ms;
  dd* ps = sm.mat + 12 * ms;
  dd* Hp = sm.mat + 13 * ms;
  dd* Gm = sm.mat + 14 * ms;
  dd* T1 = sm.mat + 15 * ms;

  // Lagrange tables and line geometry (Section 3 preamble)
  for (int t = tid; t < ng * pp; t += nt) {
    const int g = t / pp, q = t - g * pp;
    sm.phi[t] = dd{a.tab[2 * (ng + g * pp + q)], a.tab[2 * (ng + g * pp + q) + 1]};
    sm.dphi[t] = dd{a.tab[2 * (ng + ng * pp + g * pp + q)], a.tab[2 * (ng + ng * pp + g * pp + q) + 1]};
    if (a.dim == 3)
      sm.dphz[t] = dd{a.tab[2 * (ng + 2 * ng * pp + g * pp + q)], a.tab[2 * (ng + 2 * ng * pp + g * pp + q) + 1]};
  }
  __syncthreads();
  const dd c2 = two_prod(a.c, a.c);
  if (a.dim == 3) {
    // face geometry: J_b rows r_b = x_b - x0, x_b,eta, x_b,zeta; b1, b2, b3 the columns of
    // J_b^{-1}: (x_eta x x_zeta, x_zeta x r_b, r_b x x_eta) / det J_b
    const double* c0 = a.centre_xy + 3 * e;
    for (int t = tid; t < L * ng; t += nt) {
      const int l = t / ng, g = t - l * ng;
      const int64_t* fn = a.line_nodes + (sm.l0 + l) * pp;
      dd r[3], xe[3], xz[3];
      for (int d = 0; d < 3; ++d) { r[d] = dd_make(0.0); xe[d] = r[d]; xz[d] = r[d]; }
      for (int q = 0; q < pp; ++q)
        for (int d = 0; d < 3; ++d) {
          const double X = a.node_xy[3 * fn[q] + d];
          r[d] = dd_add(r[d], dd_mul_d(sm.phi[g * pp + q], X));
          xe[d] = dd_add(xe[d], dd_mul_d(sm.dphi[g * pp + q], X));
          xz[d] = dd_add(xz[d], dd_mul_d(sm.dphz[g * pp + q], X));
        }
      for (int d = 0; d < 3; ++d) r[d] = dd_sub(r[d], dd_make(c0[d]));
      auto cross = [](const dd* u, const dd* v, dd* out) {
        out[0] = dd_sub(dd_mul(u[1], v[2]), dd_mul(u[2], v[1]));
        out[1] = dd_sub(dd_mul(u[2], v[0]), dd_mul(u[0], v[2]));
        out[2] = dd_sub(dd_mul(u[0], v[1]), dd_mul(u[1], v[0]));
      };
      auto dot = [](const dd* u, const dd* v) { return dd_add(dd_add(dd_mul(u[0], v[0]), dd_mul(u[1], v[1])), dd_mul(u[2], v[2])); };
      dd n1[3], n2[3], n3[3];
      cross(xe, xz, n1);
      cross(xz, r, n2);
      cross(r, xe, n3);
      const dd det = dot(r, n1);
      const dd inv = dd_div(dd_make(1.0), det);
      dd b1[3], b2[3], b3[3];
      for (int d = 0; d < 3; ++d) { b1[d] = dd_mul(n1[d], inv); b2[d] = dd_mul(n2[d], inv); b3[d] = dd_mul(n3[d], inv); }
      const dd w = dd{a.tab[2 * g], a.tab[2 * g + 1]};
      const dd wd = dd_mul(w, det);
      const dd wdc = dd_mul(wd, c2);
      dd* K = sm.K + (l * ng + g) * 7;
      K[0] = dd_mul(wdc, dot(b1, b1));
      K[1] = dd_mul(wdc, dot(b2, b1));
      K[2] = dd_mul(wdc, dot(b3, b1));
      K[3] = dd_mul(wdc, dot(b2, b2));
      K[4] = dd_mul(wdc, dot(b2, b3));
      K[5] = dd_mul(wdc, dot(b3, b3));
      K[6] = wd;
    }
  }
  const double x0 = a.centre_xy[(size_t)a.dim * e], y0 = a.centre_xy[(size_t)a.dim * e + 1];
  for (int t = tid; a.dim == 2 && t < L * ng; t += nt) {
    const int l = t / ng, g = t - l * ng;
    const int64_t* ln = a.line_nodes + (sm.l0 + l) * pp;
    dd xb = dd_make(0.0), yb = xb, xe = xb, ye = xb;
    for (int q = 0; q < pp; ++q) {
      const double nx = a.node_xy[2 * ln[q]], ny = a.node_xy[2 * ln[q] + 1];
      xb = dd_add(xb, dd_mul_d(sm.phi[g * pp + q], nx));
      yb = dd_add(yb, dd_mul_d(sm.phi[g * pp + q], ny));
      xe = dd_add(xe, dd_mul_d(sm.dphi[g * pp + q], nx));
      ye = dd_add(ye, dd_mul_d(sm.dphi[g * pp + q], ny));
    }
    const dd rx = dd_sub(xb, dd_make(x0)), ry = dd_sub(yb, dd_make(y0));
    const dd det = dd_sub(dd_mul(rx, ye), dd_mul(ry, xe));       // det J_b
    // b1 = (y_b,eta, -x_b,eta)/det, b2 = (-(y_b - y0), x_b - x0)/det
    const dd b1x = dd_div(ye, det), b1y = dd_div(dd_neg(xe), det);
    const dd b2x = dd_div(dd_neg(ry), det), b2y = dd_div(rx, det);
    const dd w = dd{a.tab[2 * g], a.tab[2 * g + 1]};
    const dd wd = dd_mul(w, det);
    const dd wdc = dd_mul(wd, c2);
    dd* K = sm.K + (l * ng + g) * 4;
    K[0] = dd_mul(wdc, dd_add(dd_mul(b1x, b1x), dd_mul(b1y, b1y)));
    K[1] = dd_mul(wdc, dd_add(dd_mul(b2x, b1x), dd_mul(b2y, b1y)));
    K[2] = dd_mul(wdc, dd_add(dd_mul(b2x, b2x), dd_mul(b2y, b2y)));
    K[3] = wd;
    if (a.kq)
      for (int k = 0; k < 4; ++k) a.kq[((e * a.L + l) * ng + g) * 4 + k] = K[k].hi;
  }
  __syncthreads();

  const dd h = a.h;
  const dd inv_h = dd_div(dd_make(1.0), h);
  const dd inv_2h = dd_div(dd_make(0.5), h);
  const dd inv_h2 = dd_mul(inv_h, inv_h);
  const int64_t matstride = 3 * nns;
  double* mats_e = a.mats + e * (int64_t)n * matstride;

  // radial window: slots of E0/E1 hold i-1, i, i+1; E2/M0 hold i, i+1
  int s_prev = 0, s_cur = 1, s_next = 2;
  int w_cur = 0, w_next = 1;
  coefficient_matrices<DDOps>(a, sm, e, 0, E0w[s_cur], E1w[s_cur], E2w[w_cur], M0w[w_cur]);
  if (a.E_out) {
    // the comparison method needs only the coefficient matrices (with a density constant
    // along xi they are the same at every radial point)
    double* out = a.E_out + e * 4 * nns;
    for (int t = tid; t < nn; t += nt) {
      const int r = t / nb, cc = t - r * nb;
      const int64_t to = (int64_t)r * nbs + cc;
      out[to] = E0w[s_cur][t].hi;
      out[nns + to] = E1w[s_cur][t].hi;
      out[2 * nns + to] = E2w[w_cur][t].hi;
      out[3 * nns + to] = M0w[w_cur][t].hi;
    }
    return;
  }
  coefficient_matrices<DDOps>(a, sm, e, 1, E0w[s_next], E1w[s_next], E2w[w_next], M0w[w_next]);

  for (int i = 0; i <= n; ++i) {
    auto point = [&](auto ops) {
      using Op = decltype(ops);
      const dd xi = dd{a.xi_hi[i], a.xi_lo[i]};
      const dd x2 = Op::mul(xi, xi);
      // blocks of row i (Eq. (discretized) with Eq. (FD); dE by one-sided differences at the ends)
      for (int t = tid; t < nn; t += nt) {
        const int r = t / nb, cc = t - r * nb, tt = cc * nb + r;
        const dd E0 = E0w[s_cur][t], E1 = E1w[s_cur][t], E1T = E1w[s_cur][tt];
        dd dE0, dE1T;
        if (i == 0) {
          dE0 = Op::mul(Op::sub(E0w[s_next][t], E0), inv_h);
          dE1T = Op::mul(Op::sub(E1w[s_next][tt], E1T), inv_h);
        } else if (i == n) {
          dE0 = Op::mul(Op::sub(E0, E0w[s_prev][t]), inv_h);
          dE1T = Op::mul(Op::sub(E1T, E1w[s_prev][tt]), inv_h);
        } else {
          dE0 = Op::mul(Op::sub(E0w[s_next][t], E0w[s_prev][t]), inv_2h);
          dE1T = Op::mul(Op::sub(E1w[s_next][tt], E1w[s_prev][tt]), inv_2h);
        }
        dd D = Op::add(Op::sub(Op::add(E0, E1T), E1), Op::mul(xi, dE0));
        if (a.dim == 3) D = Op::add(D, E0);                   // 3-D: 2 E0 + E1^T - E1 + xi dE0
        const dd a2 = Op::mul(Op::mul(x2, E0), inv_h2);
        const dd a1 = Op::mul(Op::mul(xi, D), inv_2h);
        th[t] = Op::sub(a2, a1);
        ps[t] = Op::add(a2, a1);
        dd f = Op::neg(Op::add(a2, a2));
        f = Op::sub(f, E2w[w_cur][t]);
        f = Op::add(f, Op::mul(xi, dE1T));
        if (a.dim == 3) f = Op::add(f, E1T);                  // 3-D: + E1^T in the u coefficient
        f = Op::sub(f, Op::mul(a.mass, Op::mul(x2, M0w[w_cur][t])));
        ph[t] = f;
      }
      __syncthreads();
      if (i == 0) {
        // row -1: theta = -xi_0 E0/(2h), phi = E1^T, psi = xi_0 E0/(2h).  rho_0 = theta_0 theta_{-1}^{-1}
        for (int t = tid; t < nn; t += nt) T1[t] = Op::mul(Op::neg(Op::mul(xi, E0w[s_cur][t])), inv_2h);
        __syncthreads();
        gj_inverse<Op>(nb, T1, Gm, sm.col, sm.piv, a.status);
        mm<Op>(nb, th, Gm, Hp);                                   // Hp <- rho_0
        if (a.xel) {
          // rho_0, and the ghost u_{-1} = u_1 + Gamma u_0 from row -1: Gamma = -theta_{-1}^{-1} E1_0^T
          double* X = a.xel + e * 6 * nns;
          for (int t = tid; t < nn; t += nt) {
            const int r = t / nb, cc = t - r * nb;
            dd g = Op::make(0.0);
            for (int k = 0; k < nb; ++k) g = Op::fma(g, Gm[r * nb + k], E1w[s_cur][cc * nb + k]);
            const int64_t to = (int64_t)r * nbs + cc;
            X[to] = Hp[t].hi;
            X[2 * nns + to] = -g.hi;
          }
          __syncthreads();
        }
        // phi_0 -= rho_0 phi_{-1}; psi_0 -= rho_0 psi_{-1}
        for (int t = tid; t < nn; t += nt) {
          const int r = t / nb, cc = t - r * nb;
          dd s1 = Op::make(0.0), s2 = Op::make(0.0);
          for (int k = 0; k < nb; ++k) {
            const dd rk = Hp[r * nb + k];
            s1 = Op::fma(s1, rk, E1w[s_cur][cc * nb + k]);               // phi_{-1}[k][c] = E1[c][k]
            s2 = Op::fma(s2, rk, Op::mul(Op::mul(xi, E0w[s_cur][k * nb + cc]), inv_2h));
          }
          T1[t] = s1;
          Gm[t] = s2;
        }
        __syncthreads();
        for (int t = tid; t < nn; t += nt) {
          ph[t] = Op::sub(ph[t], T1[t]);
          ps[t] = Op::sub(ps[t], Gm[t]);
        }
        __syncthreads();
      } else {
        if (i == n && a.xel) {
          // the unmodified phi_n, for the ghost u_{n+1} (the next-point window slot is free at i = n)
          for (int t = tid; t < nn; t += nt) E0w[s_next][t] = ph[t];
          __syncthreads();
        }
        // Thomas sweep: phi_i -= theta_i phi_{i-1}^{-1} psi_{i-1} = theta_i H_{i-1}
        mm<Op>(nb, th, Hp, T1);
        for (int t = tid; t < nn; t += nt) ph[t] = Op::sub(ph[t], T1[t]);
        __syncthreads();
      }
      if (i < n) {
        gj_inverse<Op>(nb, ph, Gm, sm.col, sm.piv, a.status);     // G_i, destroys ph
        if (a.xops) {
          double* Gi = a.xops + (e * (int64_t)n + i) * nns;
          for (int t = tid; t < nn; t += nt) Gi[(int64_t)(t / nb) * nbs + (t % nb)] = Gm[t].hi;
        }
        double* Pi = mats_e + (int64_t)i * matstride;
        for (int t = tid; t < nn; t += nt) {
          const int r = t / nb, cc = t - r * nb;
          dd sp = Op::make(0.0), sq = Op::make(0.0), sh = Op::make(0.0);
          for (int k = 0; k < nb; ++k) {
            const dd gk = Gm[r * nb + k];
            sp = Op::fma(sp, gk, M0w[w_cur][k * nb + cc]);
            sq = Op::fma(sq, gk, th[k * nb + cc]);
            sh = Op::fma(sh, gk, ps[k * nb + cc]);
          }
          sp = Op::mul(sp, x2);
          const int64_t to = (int64_t)r * nbs + cc;
          Pi[to] = sp.hi;
          Pi[nns + to] = (i == 0) ? 0.0 : sq.hi;
          Pi[2 * nns + to] = sh.hi;
          T1[t] = sh;                                         // H_i kept in double-double
        }
        __syncthreads();
        for (int t = tid; t < nn; t += nt) Hp[t] = T1[t];
        __syncthreads();
      } else {
        // i == n: th = theta_n, ph = modified phi_n, ps = psi_n, Hp = H_{n-1}
        for (int t = tid; t < nn; t += nt) T1[t] = ps[t];
        __syncthreads();
        gj_inverse<Op>(nb, T1, Gm, sm.col, sm.piv, a.status);     // Gm = psi_n^{-1}
        // W = psi_{n+1} psi_n^{-1}, psi_{n+1} = xi_n E0_n / (2h)
        for (int t = tid; t < nn; t += nt) {
          const int r = t / nb, cc = t - r * nb;
          dd s = Op::make(0.0);
          for (int k = 0; k < nb; ++k)
            s = Op::fma(s, Op::mul(Op::mul(xi, E0w[s_cur][r * nb + k]), inv_2h), Gm[k * nb + cc]);
          T1[t] = s;
        }
        __syncthreads();
        if (a.xel) {
          // W, and the ghost u_{n+1} from the unmodified row n:
          // u_{n+1} = -(Y_theta u_{n-1} + Y_phi u_n - Y_M u''_n), Y_X = psi_n^{-1} X with
          // X = theta_n, the stiffness part of phi_n (phi_n + xi_n^2 M0_n / (beta dt^2)), xi_n^2 M0_n
          double* X = a.xel + e * 6 * nns;
          for (int t = tid; t < nn; t += nt) {
            const int r = t / nb, cc = t - r * nb;
            dd yt = Op::make(0.0), yp = Op::make(0.0), ym = Op::make(0.0);
            for (int k = 0; k < nb; ++k) {
              const dd gk = Gm[r * nb + k];
              const dd mk = Op::mul(x2, M0w[w_cur][k * nb + cc]);
              yt = Op::fma(yt, gk, th[k * nb + cc]);
              yp = Op::fma(yp, gk, Op::add(E0w[s_next][k * nb + cc], Op::mul(a.mass, mk)));
              ym = Op::fma(ym, gk, mk);
            }
            const int64_t to = (int64_t)r * nbs + cc;
            X[nns + to] = T1[t].hi;
            X[3 * nns + to] = yt.hi;
            X[4 * nns + to] = yp.hi;
            X[5 * nns + to] = ym.hi;
          }
          __syncthreads();
        }
        // phi_{n+1} modified = E1_n^T - theta_{n+1} H_{n-1}, theta_{n+1} = -xi_n E0_n/(2h)
        for (int t = tid; t < nn; t += nt) {
          const int r = t / nb, cc = t - r * nb;
          dd s = E1w[s_cur][cc * nb + r];
          for (int k = 0; k < nb; ++k)
            s = Op::add(s, Op::mul(Op::mul(Op::mul(xi, E0w[s_cur][r * nb + k]), inv_2h), Hp[k * nb + cc]));
          Gm[t] = s;
        }
        __syncthreads();
        double* Se = a.S + e * nns;
        double* Re = a.rt + e * 2 * nns;
        for (int t = tid; t < nn; t += nt) {
          const int r = t / nb, cc = t - r * nb;
          dd s = Gm[t], rr = Op::mul(Op::mul(xi, E0w[s_cur][t]), inv_2h), tt = Op::make(0.0);  // -theta_{n+1} = xi E0/(2h)
          for (int k = 0; k < nb; ++k) {
            const dd wk = T1[r * nb + k];
            s = Op::sub(s, Op::mul(wk, ph[k * nb + cc]));
            rr = Op::fma(rr, wk, th[k * nb + cc]);
            tt = Op::fma(tt, wk, M0w[w_cur][k * nb + cc]);
          }
          const int64_t to = (int64_t)r * nbs + cc;
          Se[to] = s.hi;
          Re[to] = rr.hi;
          Re[nns + to] = Op::mul(tt, x2).hi;
        }
        __syncthreads();
      }
    };
    if (i < kExtendedRows) point(DDOps{});
    else point(F64Ops{});
    // advance the radial window
    if (i + 1 <= n) {
      const int old_prev = s_prev;
      s_prev = s_cur;
      s_cur = s_next;
      s_next = old_prev;
      const int ow = w_cur;
      w_cur = w_next;
      w_next = ow;
      if (i + 2 <= n) {
        if (i + 2 < kExtendedPoints)
          coefficient_matrices<DDOps>(a, sm, e, i + 2, E0w[s_next], E1w[s_next], E2w[w_next], M0w[w_next]);
        else
          coefficient_matrices<F64Ops>(a, sm, e, i + 2, E0w[s_next], E1w[s_next], E2w[w_next], M0w[w_next]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 3. multifrontal factorisation of the global matrix (FP64)
// ---------------------------------------------------------------------------
struct FactorArgs {
  const TreeNodeDev* nodes;
  const int32_t* level_nodes;   // tree nodes of this level
  const int32_t* map0;
  const int32_t* map1;
  const double* S;              // [E][nb][nb]
  int nb;
  double* F;                    // workspace fronts
  double* U;                    // workspace update matrices
  double* factors;
  int* status;
  int products;                 // 1: front_factor_kernel also forms G, C and U (else front_gemm_kernel)
  int big_s;                    // > 0: fronts with s >= big_s are inverted by front_invert_grid_kernel
};

__global__ void front_assemble_kernel(FactorArgs a) {
  const TreeNodeDev nd = a.nodes[a.level_nodes[blockIdx.x]];
  const int f = nd.s + nd.b;
  double* F = a.F + nd.F_off;
  const int32_t* m0 = a.map0 + nd.map_off;
  const int32_t* m1 = a.map1 + nd.map_off;
  for (int64_t t = threadIdx.x; t < (int64_t)f * f; t += blockDim.x) {
    const int r = (int)(t / f), c = (int)(t - (int64_t)r * f);
    double v;
    if (nd.elem >= 0) {
      v = a.S[(int64_t)nd.elem * a.nb * a.nb + m0[r] * a.nb + m0[c]];
    } else {
      v = 0.0;
      const TreeNodeDev c0 = a.nodes[nd.child0], c1 = a.nodes[nd.child1];
      if (m0[r] >= 0 && m0[c] >= 0) v += a.U[c0.U_off + (int64_t)m0[r] * c0.b + m0[c]];
      if (m1[r] >= 0 && m1[c] >= 0) v += a.U[c1.U_off + (int64_t)m1[r] * c1.b + m1[c]];
    }
    F[t] = v;
  }
}

// block-wide argmax of |v| over rows k..s-1 of column k (smallest index on ties)
__device__ int block_pivot(const double* F, int f, int k, int s, double* redv, int* redi) {
  const int tid = threadIdx.x;
  double bv = -1.0;
  int bi = s;
  for (int r = k + tid; r < s; r += blockDim.x) {
    const double v = fabs(F[(int64_t)r * f + k]);
    if (v > bv) { bv = v; bi = r; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, bv, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  const int w = tid >> 5, lane = tid & 31;
  if (lane == 0) { redv[w] = bv; redi[w] = bi; }
  __syncthreads();
  if (tid == 0) {
    for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
      if (redv[j] > redv[0] || (redv[j] == redv[0] && redi[j] < redi[0])) { redv[0] = redv[j]; redi[0] = redi[j]; }
  }
  __syncthreads();
  const int r = redi[0];
  const double v = redv[0];
  __syncthreads();
  return (v > 0.0 && isfinite(v)) ? r : -1;
}

__global__ void front_factor_kernel(FactorArgs a) {
  __shared__ double redv[32];
  __shared__ int redi[32];
  __shared__ double colbuf[1024];
  const TreeNodeDev nd = a.nodes[a.level_nodes[blockIdx.x]];
  const int s = nd.s, b = nd.b, f = s + b;
  double* F = a.F + nd.F_off;
  double* X = a.factors + nd.X_off;            // s x s
  double* G = X + (int64_t)s * s;              // s x b
  double* C = G + (int64_t)s * b;              // b x s
  double* U = a.U + nd.U_off;                  // b x b
  const int tid = threadIdx.x, nt = blockDim.x;
  if (a.big_s > 0 && s >= a.big_s) return;     // inverted over the whole grid; products by tiles
  if (s > 0) {
    // X = F11^{-1}: Gauss-Jordan on [F11 | I] with row pivoting inside F11
    for (int64_t t = tid; t < (int64_t)s * s; t += nt) X[t] = ((t / s) == (t % s)) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < s; ++k) {
      const int pr = block_pivot(F, f, k, s, redv, redi);
      if (pr < 0) {
        if (tid == 0) atomicCAS(a.status, 0, SBFWI_ESINGULAR);
        return;
      }
      if (pr != k) {
        for (int c = tid; c < s; c += nt) {
          double t1 = F[(int64_t)k * f + c]; F[(int64_t)k * f + c] = F[(int64_t)pr * f + c]; F[(int64_t)pr * f + c] = t1;
          double t2 = X[(int64_t)k * s + c]; X[(int64_t)k * s + c] = X[(int64_t)pr * s + c]; X[(int64_t)pr * s + c] = t2;
        }
        __syncthreads();
      }
      const double pinv = 1.0 / F[(int64_t)k * f + k];
      // normalise row k (columns 0..s-1 of F11 and of X)
      for (int c = tid; c < s; c += nt) {
        F[(int64_t)k * f + c] *= pinv;
        X[(int64_t)k * s + c] *= pinv;
      }
      __syncthreads();
      // eliminate column k from the other rows, in chunks of the factor column
      for (int r0 = 0; r0 < s; r0 += 1024) {
        const int rn = min(1024, s - r0);
        for (int r = tid; r < rn; r += nt) colbuf[r] = (r0 + r == k) ? 0.0 : F[(int64_t)(r0 + r) * f + k];
        __syncthreads();
        for (int64_t t = tid; t < (int64_t)rn * s; t += nt) {
          const int r = (int)(t / s), c = (int)(t - (int64_t)r * s);
          const double fr = colbuf[r];
          if (fr != 0.0) {
            F[(int64_t)(r0 + r) * f + c] -= fr * F[(int64_t)k * f + c];
            X[(int64_t)(r0 + r) * s + c] -= fr * X[(int64_t)k * s + c];
          }
        }
        __syncthreads();
      }
    }
    if (!a.products) return;
    // G = X F12 (s x b), C = F21 X (b x s)
    for (int64_t t = tid; t < (int64_t)s * b; t += nt) {
      const int r = (int)(t / b), c = (int)(t - (int64_t)r * b);
      double acc = 0.0;
      for (int k = 0; k < s; ++k) acc = fma(X[(int64_t)r * s + k], F[(int64_t)k * f + s + c], acc);
      G[t] = acc;
    }
    for (int64_t t = tid; t < (int64_t)b * s; t += nt) {
      const int r = (int)(t / s), c = (int)(t - (int64_t)r * s);
      double acc = 0.0;
      for (int k = 0; k < s; ++k) acc = fma(F[(int64_t)(s + r) * f + k], X[(int64_t)k * s + c], acc);
      C[t] = acc;
    }
    __syncthreads();
  }
  if (!a.products) return;
  // update matrix U = F22 - C F12 (b x b)
  for (int64_t t = tid; t < (int64_t)b * b; t += nt) {
    const int r = (int)(t / b), c = (int)(t - (int64_t)r * b);
    double acc = F[(int64_t)(s + r) * f + s + c];
    for (int k = 0; k < s; ++k) acc = fma(-C[(int64_t)r * s + k], F[(int64_t)k * f + s + c], acc);
    U[t] = acc;
  }
}

// X = F11^{-1} of one large front by the Gauss-Jordan elimination of front_factor_kernel
// spread over the whole grid (cooperative launch, every block co-resident): per pivot, block
// 0 picks the pivot row (largest |entry|, the smallest row on ties, as block_pivot),
// swaps and normalises it; after a grid barrier every block eliminates the pivot column
// from its rows (rows blockIdx.x + k gridDim.x), reading the column before any of its
// entries change; a second barrier ends the step.  Each entry sees the operations of the
// one-block elimination in the same order, so X is the same bits.  Values written by other
// blocks are read through L2 (__ldcg).  Every barrier wait is bounded (status).
struct InvertArgs {
  FactorArgs f;
  int32_t node;
  unsigned* bar;              // [2] barrier count and generation, zero at launch
  long long budget;           // clock cycles per barrier wait
};

__global__ void __launch_bounds__(512) front_invert_grid_kernel(InvertArgs ia) {
  __shared__ double redv[32];
  __shared__ int redi[32];
  __shared__ double colv[64];
  const FactorArgs& a = ia.f;
  const TreeNodeDev nd = a.nodes[ia.node];
  const int s = nd.s, f = nd.s + nd.b;
  double* F = a.F + nd.F_off;
  double* X = a.factors + nd.X_off;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * nt + tid; t < (int64_t)s * s; t += (int64_t)gridDim.x * nt)
    X[t] = ((t / s) == (t % s)) ? 1.0 : 0.0;
  if (!grid_barrier(ia.bar, ia.bar + 1, a.status, ia.budget)) return;
  for (int k = 0; k < s; ++k) {
    if (blockIdx.x == 0) {
      double bv = -1.0;
      int bi = s;
      for (int r = k + tid; r < s; r += nt) {
        const double v = fabs(__ldcg(F + (int64_t)r * f + k));
        if (v > bv) { bv = v; bi = r; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if ((tid & 31) == 0) { redv[tid >> 5] = bv; redi[tid >> 5] = bi; }
      __syncthreads();
      if (tid == 0) {
        for (int j = 1; j < nt / 32; ++j)
          if (redv[j] > redv[0] || (redv[j] == redv[0] && redi[j] < redi[0])) { redv[0] = redv[j]; redi[0] = redi[j]; }
      }
      __syncthreads();
      const int pr = (redv[0] > 0.0 && isfinite(redv[0])) ? redi[0] : -1;
      if (pr < 0) {
        if (tid == 0) atomicCAS(a.status, 0, SBFWI_ESINGULAR);
      } else {
        if (pr != k)
          for (int c = tid; c < s; c += nt) {
            const double t1 = __ldcg(F + (int64_t)k * f + c), t2 = __ldcg(F + (int64_t)pr * f + c);
            const double x1 = __ldcg(X + (int64_t)k * s + c), x2 = __ldcg(X + (int64_t)pr * s + c);
            F[(int64_t)k * f + c] = t2; F[(int64_t)pr * f + c] = t1;
            X[(int64_t)k * s + c] = x2; X[(int64_t)pr * s + c] = x1;
          }
        __syncthreads();
        const double pinv = 1.0 / __ldcg(F + (int64_t)k * f + k);
        __syncthreads();
        for (int c = tid; c < s; c += nt) {
          F[(int64_t)k * f + c] = __ldcg(F + (int64_t)k * f + c) * pinv;
          X[(int64_t)k * s + c] = __ldcg(X + (int64_t)k * s + c) * pinv;
        }
      }
    }
    if (!grid_barrier(ia.bar, ia.bar + 1, a.status, ia.budget)) return;
    if (*(volatile int*)a.status != 0) return;        // a singular pivot: every block stops here
    // this block's rows, in groups of up to 64: the pivot-column entries first, then the rows
    for (int g0 = blockIdx.x; g0 < s; g0 += 64 * gridDim.x) {
      for (int i = tid; i < 64; i += nt) {
        const int r = g0 + i * gridDim.x;
        colv[i] = (r < s && r != k) ? __ldcg(F + (int64_t)r * f + k) : 0.0;
      }
      __syncthreads();
      for (int i = 0; i < 64; ++i) {
        const int r = g0 + i * gridDim.x;
        if (r >= s) break;
        const double fr = colv[i];
        if (fr == 0.0) continue;
        for (int c = tid; c < s; c += nt) {
          F[(int64_t)r * f + c] -= fr * __ldcg(F + (int64_t)k * f + c);
          X[(int64_t)r * s + c] -= fr * __ldcg(X + (int64_t)k * s + c);
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(ia.bar, ia.bar + 1, a.status, ia.budget)) return;
  }
}

constexpr int kGridInvertS = 192;     // separators from this size up are inverted over the whole grid

// The products of front_factor_kernel as 32 x 32 output tiles spread over many blocks (a
// level's large fronts would otherwise each keep one SM busy): item {node, kind, r0, c0},
// kind 0: G = X F12 (s x b), 1: C = F21 X (b x s), 2: U = F22 - C F12 (b x b).  Every
// output sums its terms in increasing k with fma, as the one-block loops do, so the factors
// are the same bits whichever kernel forms them.
__global__ void __launch_bounds__(256) front_gemm_kernel(FactorArgs a, const int4* items) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int4 it = items[blockIdx.x];
  const TreeNodeDev nd = a.nodes[it.x];
  const int s = nd.s, b = nd.b, f = s + b;
  const double* F = a.F + nd.F_off;
  double* X = a.factors + nd.X_off;
  double* G = X + (int64_t)s * s;
  double* C = G + (int64_t)s * b;
  double* U = a.U + nd.U_off;
  const int kind = it.y, r0 = it.z, c0 = it.w;
  const int M = kind == 0 ? s : b, N = kind == 1 ? s : b;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 8 * j, c = c0 + tx;
    acc[j] = (kind == 2 && r < M && c < N) ? F[(int64_t)(s + r) * f + s + c] : 0.0;
  }
  for (int k0 = 0; k0 < s; k0 += 32) {
    for (int t = threadIdx.x; t < 32 * 32; t += 256) {
      const int i = t >> 5, j = t & 31;
      const int r = r0 + i, k = k0 + j;          // A(r, k)
      double av = 0.0;
      if (r < M && k < s)
        av = kind == 0 ? X[(int64_t)r * s + k] : kind == 1 ? F[(int64_t)(s + r) * f + k] : -C[(int64_t)r * s + k];
      As[i][j] = av;
      const int kb = k0 + i, c = c0 + j;         // B(k, c)
      double bv = 0.0;
      if (kb < s && c < N) bv = kind == 1 ? X[(int64_t)kb * s + c] : F[(int64_t)kb * f + s + c];
      Bs[i][j] = bv;
    }
    __syncthreads();
    const int kn = min(32, s - k0);
    for (int kk = 0; kk < kn; ++kk) {
      const double bv = Bs[kk][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fma(As[ty + 8 * j][kk], bv, acc[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 8 * j, c = c0 + tx;
    if (r >= M || c >= N) continue;
    if (kind == 0) G[(int64_t)r * b + c] = acc[j];
    else if (kind == 1) C[(int64_t)r * s + c] = acc[j];
    else U[(int64_t)r * b + c] = acc[j];
  }
}

// Factors of the transposed global matrix from those of the matrix: the front of a tree node
// for A^T is the transpose of its front for A, so X' = F11^{-T} = X^T, G' = X' F21^T = C^T and
// C' = F12^T X' = G^T (same storage layout: X' s x s, G' s x b, C' b x s).  One block per node.
__global__ void transpose_factors_kernel(const TreeNodeDev* nodes, int n_nodes, const double* f, double* ft) {
  for (int v = blockIdx.x; v < n_nodes; v += gridDim.x) {
    const TreeNodeDev nd = nodes[v];
    const int s = nd.s, b = nd.b;
    if (s == 0) continue;
    const double* X = f + nd.X_off;
    const double* G = X + (int64_t)s * s;
    const double* C = G + (int64_t)s * b;
    double* Xt = ft + nd.X_off;
    double* Gt = Xt + (int64_t)s * s;
    double* Ct = Gt + (int64_t)s * b;
    for (int64_t t = threadIdx.x; t < (int64_t)s * s; t += blockDim.x) {
      const int r = (int)(t / s), c = (int)(t - (int64_t)r * s);
      Xt[t] = X[(int64_t)c * s + r];
    }
    for (int64_t t = threadIdx.x; t < (int64_t)s * b; t += blockDim.x) {     // G'[r][c] = C[c][r], r < s, c < b
      const int r = (int)(t / b), c = (int)(t - (int64_t)r * b);
      Gt[t] = C[(int64_t)c * s + r];
    }
    for (int64_t t = threadIdx.x; t < (int64_t)b * s; t += blockDim.x) {     // C'[r][c] = G[c][r], r < b, c < s
      const int r = (int)(t / s), c = (int)(t - (int64_t)r * s);
      Ct[t] = G[(int64_t)c * b + r];
    }
  }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
template <class T>
static int upload(DevBuf& d, const std::vector<T>& h, cudaStream_t st) {
  SBFWI_CUDA(d.alloc(sizeof(T) * h.size()));
  if (!h.empty()) SBFWI_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
  return SBFWI_OK;
}

static int read_status(const DevBuf& st_dev, cudaStream_t st, int* code) {
  SBFWI_CUDA(cudaMemcpyAsync(code, st_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SBFWI_CUDA(cudaStreamSynchronize(st));
  return SBFWI_OK;
}

// mesh-only device data (first set-up on a mesh, or after a device change)
static int ensure_mesh_device(const Mesh& m, cudaStream_t st) {
  int device = 0;
  SBFWI_CUDA(cudaGetDevice(&device));
  if (m.dev && m.dev->device == device) return SBFWI_OK;
  auto d = std::make_unique<MeshDevice>();
  d->device = device;
  const int n = m.n, p = m.p, pp = p + 1;
  const int ng = (3 * p + 2) / 2;
  const int ng1 = (3 * p + 4) / 2;          // 3-D: points per direction of the tensor face rule
  // radial grid xi_i = xi0 + i h (xi_n = 1), double-double
  std::vector<double> xi_hi(n + 1), xi_lo(n + 1);
  const dd h = dd_div(dd_sub(dd_make(1.0), dd_make(m.xi0)), dd_make((double)n));
  for (int i = 0; i <= n; ++i) {
    dd x = (i == n) ? dd_make(1.0) : dd_add(dd_make(m.xi0), dd_mul_d(h, (double)i));
    xi_hi[i] = x.hi; xi_lo[i] = x.lo;
  }
  // Gauss rule and Lagrange tables.  2-D lines: ng points, phi and dphi of the p+1 line
  // nodes.  3-D faces: the tensor rule of ng1^2 points (point ga + ng1 gb at (eta_ga,
  // zeta_gb)), N, N_eta and N_zeta of the (p+1)^2 face nodes (node a + (p+1) b)
  std::vector<double> tab;
  if (m.dim == 3) {
    std::vector<dd> gx_, gw_;
    gauss_legendre_dd(ng1, gx_, gw_);
    const int G = ng1 * ng1, F = pp * pp;
    tab.assign(2 * (G + 3 * G * F), 0.0);
    std::vector<dd> ph(pp * ng1), dph(pp * ng1);
    for (int g = 0; g < ng1; ++g) lagrange_dd(p, gx_[g], ph.data() + g * pp, dph.data() + g * pp);
    auto put = [&](size_t k, dd v) { tab[2 * k] = v.hi; tab[2 * k + 1] = v.lo; };
    for (int gb = 0; gb < ng1; ++gb)
      for (int ga = 0; ga < ng1; ++ga) {
        const int g = ga + ng1 * gb;
        put(g, dd_mul(gw_[ga], gw_[gb]));
        for (int b = 0; b < pp; ++b)
          for (int a2 = 0; a2 < pp; ++a2) {
            const int q = a2 + pp * b;
            put(G + (size_t)g * F + q, dd_mul(ph[ga * pp + a2], ph[gb * pp + b]));
            put(G + (size_t)G * F + (size_t)g * F + q, dd_mul(dph[ga * pp + a2], ph[gb * pp + b]));
            put(G + 2 * (size_t)G * F + (size_t)g * F + q, dd_mul(ph[ga * pp + a2], dph[gb * pp + b]));
          }
      }
  } else {
    std::vector<dd> gx_, gw_;
    gauss_legendre_dd(ng, gx_, gw_);
    tab.assign(2 * (ng + 2 * ng * pp), 0.0);
    for (int g = 0; g < ng; ++g) {
      tab[2 * g] = gw_[g].hi; tab[2 * g + 1] = gw_[g].lo;
      std::vector<dd> ph(pp), dph(pp);
      lagrange_dd(p, gx_[g], ph.data(), dph.data());
      for (int q = 0; q < pp; ++q) {
        tab[2 * (ng + g * pp + q)] = ph[q].hi; tab[2 * (ng + g * pp + q) + 1] = ph[q].lo;
        tab[2 * (ng + ng * pp + g * pp + q)] = dph[q].hi; tab[2 * (ng + ng * pp + g * pp + q) + 1] = dph[q].lo;
      }
    }
  }
  int rc;
  if ((rc = upload(d->xy, m.node_xy, st))) return rc;
  if ((rc = upload(d->ctr, m.centre_xy, st))) return rc;
  if ((rc = upload(d->lines, m.line_nodes, st))) return rc;
  if ((rc = upload(d->lloc, m.line_local, st))) return rc;
  if ((rc = upload(d->dofs, m.dofs, st))) return rc;
  if ((rc = upload(d->nbe, m.nbe, st))) return rc;
  if ((rc = upload(d->lptr, m.elem_ptr, st))) return rc;
  if (m.uneven && (rc = upload(d->api_map, m.api_to_lib, st))) return rc;
  if ((rc = upload(d->xih, xi_hi, st))) return rc;
  if ((rc = upload(d->xil, xi_lo, st))) return rc;
  if ((rc = upload(d->tab, tab, st))) return rc;
  const Tree& t = m.tree;
  if ((rc = upload(d->tree_nodes, t.nodes, st))) return rc;
  if ((rc = upload(d->sep_nodes, t.sep_nodes, st))) return rc;
  if ((rc = upload(d->bnd_nodes, t.bnd_nodes, st))) return rc;
  if ((rc = upload(d->map0, t.map0, st))) return rc;
  if ((rc = upload(d->map1, t.map1, st))) return rc;
  if ((rc = upload(d->src0, t.src0, st))) return rc;
  if ((rc = upload(d->src1, t.src1, st))) return rc;
  std::vector<int32_t> all;
  for (int l = 0; l < t.levels; ++l) {
    d->level_start.push_back((int64_t)all.size());
    all.insert(all.end(), t.nodes_at_level[l].begin(), t.nodes_at_level[l].end());
  }
  if ((rc = upload(d->level_nodes, all, st))) return rc;
  // tiles of the front products for the levels with fewer fronts than SMs: per level
  // [G and C tiles | U tiles], offsets fgemm_start[3l .. 3l+2]
  {
    int sms = 152;
    int dev_id = 0;
    if (cudaGetDevice(&dev_id) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    std::vector<int4> items;
    for (int l = 0; l < t.levels; ++l) {
      const bool tiled = (int)t.nodes_at_level[l].size() < sms;
      d->fgemm_level.push_back(tiled ? 1 : 0);
      d->fgemm_start.push_back((int64_t)items.size());
      if (tiled)
        for (int32_t nd : t.nodes_at_level[l]) {
          const TreeNodeDev& r = t.nodes[nd];
          if (r.s == 0 || r.b == 0) continue;
          for (int r0 = 0; r0 < r.s; r0 += 32)
            for (int c0 = 0; c0 < r.b; c0 += 32) items.push_back(make_int4(nd, 0, r0, c0));
          for (int r0 = 0; r0 < r.b; r0 += 32)
            for (int c0 = 0; c0 < r.s; c0 += 32) items.push_back(make_int4(nd, 1, r0, c0));
        }
      d->fgemm_start.push_back((int64_t)items.size());
      if (tiled)
        for (int32_t nd : t.nodes_at_level[l]) {
          const TreeNodeDev& r = t.nodes[nd];
          for (int r0 = 0; r0 < r.b; r0 += 32)
            for (int c0 = 0; c0 < r.b; c0 += 32) items.push_back(make_int4(nd, 2, r0, c0));
        }
      d->fgemm_start.push_back((int64_t)items.size());
    }
    if (items.empty()) items.push_back(make_int4(0, 0, 0, 0));
    if ((rc = upload(d->fgemm, items, st))) return rc;
  }
  SBFWI_CUDA(d->F.alloc(sizeof(double) * std::max<int64_t>(t.F_total, 1)));
  SBFWI_CUDA(d->U.alloc(sizeof(double) * std::max<int64_t>(t.U_total, 1)));
  SBFWI_CUDA(cudaStreamSynchronize(st));     // host vectors above go out of scope
  m.dev = std::move(d);
  return SBFWI_OK;
}

// base cell, clamping and transpose CSR of the bilinear (3-D: trilinear) map for one
// fine grid
static int ensure_grid_map(const Mesh& m, int64_t gx, int64_t gy, int64_t gz, double lx, double ly, double lz,
                           cudaStream_t st) {
  MeshDevice& d = *m.dev;
  if (d.grid_ready && d.gx == gx && d.gy == gy && d.gz == gz && d.lx == lx && d.ly == ly && d.lz == lz) return SBFWI_OK;
  d.grid_ready = false;
  const int n = m.n, nb = m.nb, D = m.dim, corners = 1 << D;
  const int64_t np = m.n_nodal;
  std::vector<int32_t> cell(np, 0);
  std::vector<int8_t> clamp(np, 0);
  const long double h = (1.0L - (long double)m.xi0) / n;
  // padding points of uneven meshes sit at their element's centre and are left out of
  // the transpose (their gradient is zero)
  auto padding = [&](int64_t q) {
    if (q >= m.n_int) return false;
    const int64_t e = q / ((int64_t)n * nb);
    return (int)(q % nb) >= m.nbe[e];
  };
  const int64_t gdim[3] = {gx, gy, gz};
  const long double len[3] = {lx, ly, lz};
  for (int64_t q = 0; q < np; ++q) {
    long double x[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) {
      if (padding(q)) {
        const int64_t e = q / ((int64_t)n * nb);
        x[k] = m.centre_xy[(size_t)D * e + k];
      } else if (q < m.n_int) {
        const int64_t e = q / ((int64_t)n * nb), rem = q - e * (int64_t)n * nb;
        const int i = (int)(rem / nb), j = (int)(rem - (int64_t)i * nb);
        const int32_t g = m.dofs[e * nb + j];
        const long double xi = (long double)m.xi0 + (long double)i * h;
        const long double c0 = m.centre_xy[(size_t)D * e + k];
        x[k] = c0 + xi * ((long double)m.node_xy[(size_t)D * g + k] - c0);
      } else {
        x[k] = m.node_xy[(size_t)D * (q - m.n_int) + k];
      }
    }
    int64_t ix[3] = {0, 0, 0};
    int8_t cl = 0;
    for (int k = 0; k < D; ++k) {
      const long double f = x[k] * gdim[k] / len[k] - 0.5L;
      ix[k] = (int64_t)std::floor(f);
      if (ix[k] < 0) { ix[k] = 0; cl |= (int8_t)(1 << (2 * k)); }
      if (ix[k] > gdim[k] - 2) { ix[k] = gdim[k] - 2; cl |= (int8_t)(2 << (2 * k)); }
    }
    cell[q] = (int32_t)((D == 3 ? ix[2] * gy : 0) * gx + ix[1] * gx + ix[0]);
    clamp[q] = cl;
  }
  // the transpose map gathers, per grid cell, the points touching it in point order
  const int64_t ncell = gx * gy * (D == 3 ? gz : 1);
  std::vector<int64_t> cnt(ncell + 1, 0);
  auto corner_cell = [&](int64_t q, int k) {
    return (int64_t)cell[q] + (k & 1) + ((k >> 1) & 1) * gx + (k >> 2) * gx * gy;
  };
  for (int64_t q = 0; q < np; ++q)
    if (!padding(q))
      for (int k = 0; k < corners; ++k) cnt[corner_cell(q, k) + 1]++;
  for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
  std::vector<int64_t> list(cnt.back());
  std::vector<int64_t> fillp(cnt.begin(), cnt.end() - 1);
  for (int64_t q = 0; q < np; ++q)
    if (!padding(q))
      for (int k = 0; k < corners; ++k) list[fillp[corner_cell(q, k)]++] = q * corners + k;
  int rc;
  if ((rc = upload(d.cell, cell, st))) return rc;
  if ((rc = upload(d.clamp, clamp, st))) return rc;
  if ((rc = upload(d.cell_ptr, cnt, st))) return rc;
  if ((rc = upload(d.cell_list, list, st))) return rc;
  SBFWI_CUDA(cudaStreamSynchronize(st));
  d.gx = gx; d.gy = gy; d.gz = gz; d.lx = lx; d.ly = ly; d.lz = lz;
  d.grid_ready = true;
  return SBFWI_OK;
}

// The nodal gradient operator of the full Frechet kernel, in the library's padded nodal
// layout: at radial point xi_i of local node j on one line element of element e,
// [u_xi; u_eta] = J [u_x; u_y] with J = [[x_b - x0, y_b - y0], [xi x_b,eta, xi y_b,eta]]
// (the coordinate map x = x0 + xi (x_b(eta) - x0)); u_xi by second-order differences on
// the radial grid (central inside, one-sided at xi_0 and xi_n = 1), u_eta by the line's
// Lagrange derivative at the node; a point met by several (element, line) pairs takes
// the mean of their gradients.
int ensure_gradient_operator(const Mesh& m, cudaStream_t st) {
  MeshDevice& d = *m.dev;
  if (d.grad_ready) return SBFWI_OK;
  const int n = m.n, nb = m.nb, p = m.p, pp = p + 1;
  const int64_t npt = m.n_nodal;
  if (npt > INT32_MAX) return fail(SBFWI_EUNSUPPORTED, "the full kernel's gradient operator needs fewer than 2^31 nodal points");
  const double h = (1.0 - m.xi0) / n;
  std::vector<double> eta(pp), D((size_t)pp * pp, 0.0);    // D[k][a] = d phi_a / d eta at node k
  for (int k = 0; k < pp; ++k) eta[k] = -1.0 + 2.0 * k / p;
  for (int a = 0; a < pp; ++a) {
    double denom = 1.0;
    for (int b = 0; b < pp; ++b) if (b != a) denom *= eta[a] - eta[b];
    for (int k = 0; k < pp; ++k) {
      double sum = 0.0;
      for (int b = 0; b < pp; ++b) {
        if (b == a) continue;
        double prod = 1.0;
        for (int c = 0; c < pp; ++c) if (c != a && c != b) prod *= eta[k] - eta[c];
        sum += prod;
      }
      D[(size_t)k * pp + a] = sum / denom;
    }
  }
  std::vector<int64_t> R;
  std::vector<int32_t> C;
  std::vector<double> V;
  std::vector<int32_t> cnt(npt, 0);
  for (int64_t e = 0; e < m.n_elem; ++e) {
    const double x0 = m.centre_xy[2 * e], y0 = m.centre_xy[2 * e + 1];
    auto idx = [&](int i, int j) -> int64_t {
      return i < n ? (e * n + i) * (int64_t)nb + j : m.n_int + m.dofs[(size_t)e * nb + j];
    };
    for (int64_t l = m.elem_ptr[e]; l < m.elem_ptr[e + 1]; ++l) {
      const int64_t* ln = m.line_nodes.data() + l * pp;
      const int32_t* loc = m.line_local.data() + l * pp;
      std::vector<double> dx(pp, 0.0), dy(pp, 0.0);
      for (int k = 0; k < pp; ++k)
        for (int a = 0; a < pp; ++a) {
          dx[k] += D[(size_t)k * pp + a] * m.node_xy[2 * ln[a]];
          dy[k] += D[(size_t)k * pp + a] * m.node_xy[2 * ln[a] + 1];
        }
      for (int i = 0; i <= n; ++i) {
        const double xi = i == n ? 1.0 : m.xi0 + i * h;
        int si[3], ns;
        double sw[3];
        if (i == 0) { si[0] = 0; si[1] = 1; si[2] = 2; sw[0] = -3; sw[1] = 4; sw[2] = -1; ns = 3; }
        else if (i == n) { si[0] = n; si[1] = n - 1; si[2] = n - 2; sw[0] = 3; sw[1] = -4; sw[2] = 1; ns = 3; }
        else { si[0] = i + 1; si[1] = i - 1; sw[0] = 1; sw[1] = -1; ns = 2; }
        for (int k = 0; k < pp; ++k) {
          const int j = loc[k];
          const double j00 = m.node_xy[2 * ln[k]] - x0, j01 = m.node_xy[2 * ln[k] + 1] - y0;
          const double j10 = xi * dx[k], j11 = xi * dy[k];
          const double det = j00 * j11 - j01 * j10;
          const double inv[2][2] = {{j11 / det, -j01 / det}, {-j10 / det, j00 / det}};
          const int64_t q = idx(i, j);
          for (int dd = 0; dd < 2; ++dd) {
            for (int t = 0; t < ns; ++t) {
              R.push_back(2 * q + dd); C.push_back((int32_t)idx(si[t], j)); V.push_back(inv[dd][0] * sw[t] / (2 * h));
            }
            for (int a = 0; a < pp; ++a) {
              R.push_back(2 * q + dd); C.push_back((int32_t)idx(i, loc[a])); V.push_back(inv[dd][1] * D[(size_t)k * pp + a]);
            }
          }
          ++cnt[q];
        }
      }
    }
  }
  std::vector<int64_t> ptr(2 * npt + 1, 0);
  for (size_t t = 0; t < R.size(); ++t) ++ptr[R[t] + 1];
  for (int64_t r = 0; r < 2 * npt; ++r) ptr[r + 1] += ptr[r];
  std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
  std::vector<int32_t> col(R.size());
  std::vector<double> val(R.size());
  for (size_t t = 0; t < R.size(); ++t) {
    const int64_t at = fill[R[t]]++;
    col[at] = C[t];
    val[at] = V[t] / cnt[R[t] / 2];
  }
  int rc;
  if ((rc = upload(d.grad_ptr, ptr, st))) return rc;
  if ((rc = upload(d.grad_col, col, st))) return rc;
  if ((rc = upload(d.grad_val, val, st))) return rc;
  SBFWI_CUDA(cudaStreamSynchronize(st));
  d.grad_ready = true;
  return SBFWI_OK;
}

// One launch sequence of the element set-up kernel (chunked when the working matrices
// live in global memory).  E_out: the comparison method's coefficient matrices only;
// xops/xel/kq: the exact adjoint's extra operators (nullable).
static int launch_element_setup(Model& md, const Mesh& m, const double* rho_hi, const double* rho_lo, double* E_out,
                                double* xops, double* xel, double* kq, int* status, cudaStream_t st) {
  const int nb = m.nb, n = m.n, p = m.p, L = m.L, pp = m.fpp;
  const int ng = m.dim == 3 ? ((3 * p + 4) / 2) * ((3 * p + 4) / 2) : (3 * p + 2) / 2;
  const int nk = m.dim == 3 ? 7 : 4;
  const int64_t E = m.n_elem, nn = (int64_t)nb * nb;
  const MeshDevice& d = *m.dev;
  Profiler& prof = profiler();
  ElemArgs a;
  a.nb = nb; a.n = n; a.L = L; a.p = p; a.ng = ng; a.n_elem = E; a.n_int = m.n_int;
  a.dim = m.dim; a.fpp = pp; a.nk = nk;
  a.nbe = d.nbe.as<int32_t>(); a.lptr = d.lptr.as<int64_t>(); a.mat_ws = nullptr; a.e0 = 0;
  a.E_out = E_out;
  a.xops = xops; a.xel = xel; a.kq = kq;
  a.c = md.c;
  a.mass = dd_div(dd_make(1.0), dd_mul(dd_make(md.beta), two_prod(md.dt, md.dt)));
  a.h = dd_div(dd_sub(dd_make(1.0), dd_make(m.xi0)), dd_make((double)n));
  a.node_xy = d.xy.as<double>(); a.centre_xy = d.ctr.as<double>();
  a.line_nodes = d.lines.as<int64_t>(); a.line_local = d.lloc.as<int32_t>(); a.dofs = d.dofs.as<int32_t>();
  a.rho_hi = rho_hi; a.rho_lo = rho_lo;
  a.xi_hi = d.xih.as<double>(); a.xi_lo = d.xil.as<double>(); a.tab = d.tab.as<double>();
  a.mats = md.mats.as<double>(); a.rt = md.rt.as<double>(); a.S = md.S.as<double>(); a.status = status;
  // the 16 working matrices live in shared memory up to n_b = 24; beyond, in a global
  // workspace, with the elements set up in chunks that bound its size
  const size_t small =
      sizeof(dd) * ((size_t)L * ng * 2 * nk + (size_t)L * pp * pp * 4 + (m.dim == 3 ? 3 : 2) * (size_t)ng * pp + nb) + 16;
  const size_t mat_bytes = sizeof(dd) * 16 * (size_t)nn;
  const bool in_smem = small + mat_bytes <= 160 * 1024;
  const size_t smem = in_smem ? small + mat_bytes : small;
  SBFWI_CUDA(cudaFuncSetAttribute(element_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaFuncAttributes fattr;
  SBFWI_CUDA(cudaFuncGetAttributes(&fattr, element_setup_kernel));
  int threads = (int)std::min<int64_t>((nn + 31) / 32 * 32, fattr.maxThreadsPerBlock / 32 * 32);
  if (threads < 64) threads = 64;
  const int64_t chunk = in_smem ? E : std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)((256u << 20) / mat_bytes)));
  DevBuf ws;
  if (!in_smem) {
    SBFWI_CUDA(ws.alloc(mat_bytes * chunk));
    a.mat_ws = ws.as<dd>();
  }
  for (int64_t e0 = 0; e0 < E; e0 += chunk) {
    a.e0 = e0;
    element_setup_kernel<<<(unsigned)std::min(chunk, E - e0), threads, smem, st>>>(a);
    prof.count(kPhaseSetup);
    SBFWI_CUDA(cudaGetLastError());
  }
  if (!in_smem) SBFWI_CUDA(cudaStreamSynchronize(st));   // the workspace is freed on return
  return SBFWI_OK;
}

int setup_model(Model& md, const Mesh& m, const double* rho, int mem, cudaStream_t st) {
  const int nb = m.nb, n = m.n;
  const int64_t E = m.n_elem, N = m.n_nodes, np = m.n_nodal;
  md.nb = nb; md.n = n; md.E = E; md.N = N;
  int rc;
  if ((rc = ensure_mesh_device(m, st))) return rc;
  if (md.rho_kind == SBFWI_RHO_GRID && (rc = ensure_grid_map(m, md.gx, md.gy, md.gz, md.lx, md.ly, md.lz, st)))
    return rc;
  const MeshDevice& d = *m.dev;
  DevBuf status;
  SBFWI_CUDA(status.alloc(sizeof(int)));
  SBFWI_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st));
  Profiler& prof = profiler();
  prof.begin(kPhaseSetup, st);

  // density input (nodal values arrive in the caller's layout; uneven meshes spread
  // them to the library's padded layout, padding points get 1)
  DevBuf d_rho_in, d_rho_api;
  const bool nodal = md.rho_kind == SBFWI_RHO_NODAL;
  const int64_t nrho = nodal ? m.n_nodal_api : md.gx * md.gy * (m.dim == 3 ? md.gz : 1);
  const cudaMemcpyKind kind = mem == SBFWI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (nodal && m.uneven) {
    SBFWI_CUDA(d_rho_api.alloc(sizeof(double) * nrho));
    SBFWI_CUDA(cudaMemcpyAsync(d_rho_api.p, rho, sizeof(double) * nrho, kind, st));
    SBFWI_CUDA(d_rho_in.alloc(sizeof(double) * np));
    const unsigned blocks = (unsigned)std::min<int64_t>((np + 255) / 256, 152 * 8);
    fill_kernel<<<blocks, 256, 0, st>>>(d_rho_in.as<double>(), np, 1.0);
    scatter_nodal_kernel<<<blocks, 256, 0, st>>>(d_rho_api.as<double>(), d.api_map.as<int64_t>(), nrho,
                                                 d_rho_in.as<double>());
    prof.count(kPhaseSetup, 2);
    SBFWI_CUDA(cudaGetLastError());
  } else {
    SBFWI_CUDA(d_rho_in.alloc(sizeof(double) * nrho));
    SBFWI_CUDA(cudaMemcpyAsync(d_rho_in.p, rho, sizeof(double) * nrho, kind, st));
  }
  DevBuf rho_hi, rho_lo;
  SBFWI_CUDA(rho_hi.alloc(sizeof(double) * np));
  SBFWI_CUDA(rho_lo.alloc(sizeof(double) * np));
  SBFWI_CUDA(md.pts_hi.alloc(sizeof(double) * m.dim * np));
  SBFWI_CUDA(md.pts_lo.alloc(sizeof(double) * m.dim * np));
  {
    DensityArgs a;
    a.n_elem = E; a.n_nodes = N; a.n_int = m.n_int; a.nb = nb; a.n = n; a.nbe = d.nbe.as<int32_t>();
    a.node_xy = d.xy.as<double>(); a.centre_xy = d.ctr.as<double>(); a.dofs = d.dofs.as<int32_t>();
    a.xi_hi = d.xih.as<double>(); a.xi_lo = d.xil.as<double>();
    a.grid = d_rho_in.as<double>(); a.rho_kind = md.rho_kind; a.dim = m.dim;
    a.gx = md.gx; a.gy = md.gy; a.gz = md.gz; a.lx = md.lx; a.ly = md.ly; a.lz = md.lz;
    a.cell_of_point = md.rho_kind == SBFWI_RHO_GRID ? d.cell.as<int32_t>() : nullptr;
    a.clamp_of_point = md.rho_kind == SBFWI_RHO_GRID ? d.clamp.as<int8_t>() : nullptr;
    a.pts_hi = md.pts_hi.as<double>(); a.pts_lo = md.pts_lo.as<double>();
    a.rho_hi = rho_hi.as<double>(); a.rho_lo = rho_lo.as<double>(); a.status = status.as<int>();
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((np + threads - 1) / threads, 152 * 32);
    if (m.dim == 3) density3d_kernel<<<blocks, threads, 0, st>>>(a);
    else density_kernel<<<blocks, threads, 0, st>>>(a);
    prof.count(kPhaseSetup);
    SBFWI_CUDA(cudaGetLastError());
  }
  SBFWI_CUDA(md.rho_nodal.alloc(sizeof(double) * np));
  SBFWI_CUDA(cudaMemcpyAsync(md.rho_nodal.p, rho_hi.p, sizeof(double) * np, cudaMemcpyDeviceToDevice, st));
  if (!md.lfe) {
    SBFWI_CUDA(md.rho_lo.alloc(sizeof(double) * np));
    SBFWI_CUDA(cudaMemcpyAsync(md.rho_lo.p, rho_lo.p, sizeof(double) * np, cudaMemcpyDeviceToDevice, st));
  }

  if (md.lfe) {
    const unsigned blocks = (unsigned)std::min<int64_t>((m.n_int + 255) / 256, 152 * 8);
    radial_constant_density_kernel<<<blocks, 256, 0, st>>>(rho_hi.as<double>(), rho_lo.as<double>(),
                                                           d.dofs.as<int32_t>(), d.nbe.as<int32_t>(), m.n_int, n, nb);
    prof.count(kPhaseSetup);
    SBFWI_CUDA(cudaGetLastError());
  }

  // element set-up
  const int64_t nn = (int64_t)nb * nb;
  // the comparison method has no radial interior: no per-point operators
  SBFWI_CUDA(md.mats.alloc(md.lfe ? 16 : sizeof(double) * E * n * 3 * nn));
  SBFWI_CUDA(md.rt.alloc(md.lfe ? 16 : sizeof(double) * E * 2 * nn));
  SBFWI_CUDA(md.S.alloc(sizeof(double) * E * nn));
  if (m.uneven) {   // rows and columns beyond an element's n_b stay zero
    SBFWI_CUDA(cudaMemsetAsync(md.mats.p, 0, md.mats.bytes, st));
    SBFWI_CUDA(cudaMemsetAsync(md.rt.p, 0, md.rt.bytes, st));
    SBFWI_CUDA(cudaMemsetAsync(md.S.p, 0, md.S.bytes, st));
  }
  {
    DevBuf E_dev;
    if (md.lfe) {
      SBFWI_CUDA(E_dev.alloc(sizeof(double) * E * 4 * nn));
      SBFWI_CUDA(cudaMemsetAsync(E_dev.p, 0, E_dev.bytes, st));
    }
    if ((rc = launch_element_setup(md, m, rho_hi.as<double>(), rho_lo.as<double>(), md.lfe ? E_dev.as<double>() : nullptr,
                                   nullptr, nullptr, nullptr, status.as<int>(), st)))
      return rc;
    if (md.lfe) {
      // the comparison method's K and M of every element on the device (lfe_setup.cu); S = K + a0 M
      // for the global system, M for the per-step effective sources
      SBFWI_CUDA(md.lfe_M.alloc(sizeof(double) * E * nn));
      SBFWI_CUDA(cudaMemsetAsync(md.lfe_M.p, 0, md.lfe_M.bytes, st));
      if ((rc = lfe_setup_device(md, E_dev.as<double>(), md.S.as<double>(), md.lfe_M.as<double>(), st))) return rc;
    }
  }

  // the per-step operators split for the tensor cores
  if (!md.lfe && tc_supported(nb, 1) && (rc = tc_prepare(md, st))) return rc;

  // global factorisation along the elimination tree
  const Tree& t = m.tree;
  {
    const size_t fb = sizeof(double) * (size_t)std::max<int64_t>(t.X_total, 1);
    const size_t nmap = t.src0.size(), nsep = t.sep_nodes.size(), nbnd = t.bnd_nodes.size();
    const size_t ib = sizeof(int32_t) * (2 * nmap + nsep + nbnd);
    SBFWI_CUDA(md.factors.alloc(fb + ib));
    int32_t* tail = reinterpret_cast<int32_t*>(md.factors.as<char>() + fb);
    md.solve_src0 = tail;
    md.solve_src1 = tail + nmap;
    md.solve_sep = tail + 2 * nmap;
    md.solve_bnd = tail + 2 * nmap + nsep;
    md.solve_bytes = fb + ib;
    if (nmap) {
      SBFWI_CUDA(cudaMemcpyAsync(tail, d.src0.p, sizeof(int32_t) * nmap, cudaMemcpyDeviceToDevice, st));
      SBFWI_CUDA(cudaMemcpyAsync(tail + nmap, d.src1.p, sizeof(int32_t) * nmap, cudaMemcpyDeviceToDevice, st));
    }
    if (nsep) SBFWI_CUDA(cudaMemcpyAsync(tail + 2 * nmap, d.sep_nodes.p, sizeof(int32_t) * nsep, cudaMemcpyDeviceToDevice, st));
    if (nbnd)
      SBFWI_CUDA(cudaMemcpyAsync(tail + 2 * nmap + nsep, d.bnd_nodes.p, sizeof(int32_t) * nbnd, cudaMemcpyDeviceToDevice, st));
  }
  {
    FactorArgs a;
    a.nodes = d.tree_nodes.as<TreeNodeDev>(); a.map0 = d.map0.as<int32_t>(); a.map1 = d.map1.as<int32_t>();
    a.S = md.S.as<double>(); a.nb = nb; a.F = d.F.as<double>(); a.U = d.U.as<double>();
    a.factors = md.factors.as<double>(); a.status = status.as<int>();
    // the grid of the cooperative inversion: one block of 512 threads per SM, as many as fit
    DevBuf inv_bar;
    SBFWI_CUDA(inv_bar.alloc(2 * sizeof(unsigned)));
    int inv_grid = 0;
    {
      int dev_id = 0, sms = 0, per_sm = 0;
      SBFWI_CUDA(cudaGetDevice(&dev_id));
      SBFWI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id));
      SBFWI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, front_invert_grid_kernel, 512, 0));
      inv_grid = std::max(1, std::min(per_sm, 1) * sms);
    }
    for (int l = 0; l < t.levels; ++l) {
      a.level_nodes = d.level_nodes.as<int32_t>() + d.level_start[l];
      const unsigned cnt = (unsigned)t.nodes_at_level[l].size();
      // the products go to the tiled kernel on levels with fewer fronts than SMs (one block
      // per front would leave most SMs idle); levels with many small fronts keep them in
      // front_factor_kernel
      const int64_t gc0 = d.fgemm_start[3 * l], u0 = d.fgemm_start[3 * l + 1], u1 = d.fgemm_start[3 * l + 2];
      a.products = d.fgemm_level[l] ? 0 : 1;
      a.big_s = d.fgemm_level[l] ? kGridInvertS : 0;
      front_assemble_kernel<<<cnt, 256, 0, st>>>(a);
      front_factor_kernel<<<cnt, 512, 0, st>>>(a);
      prof.count(kPhaseSetup, 2);
      if (a.big_s > 0)
        for (int32_t v : t.nodes_at_level[l]) {
          if (t.nodes[v].s < kGridInvertS) continue;
          InvertArgs ia;
          ia.f = a; ia.node = v; ia.bar = inv_bar.as<unsigned>(); ia.budget = 4000000000LL;
          SBFWI_CUDA(cudaMemsetAsync(inv_bar.p, 0, inv_bar.bytes, st));
          void* kargs[] = {&ia};
          SBFWI_CUDA(cudaLaunchCooperativeKernel((const void*)front_invert_grid_kernel, dim3(inv_grid), dim3(512), kargs,
                                                 0, st));
          prof.count(kPhaseSetup);
        }
      if (!a.products) {
        const int4* items = d.fgemm.as<int4>();
        if (u0 > gc0) { front_gemm_kernel<<<(unsigned)(u0 - gc0), 256, 0, st>>>(a, items + gc0); prof.count(kPhaseSetup); }
        if (u1 > u0) { front_gemm_kernel<<<(unsigned)(u1 - u0), 256, 0, st>>>(a, items + u0); prof.count(kPhaseSetup); }
      }
      SBFWI_CUDA(cudaGetLastError());
    }
  }
  prof.end(kPhaseSetup, st);
  int code = 0;
  if ((rc = read_status(status, st, &code))) return rc;
  if (code == SBFWI_EINVAL) return fail(SBFWI_EINVAL, "density must be positive at every nodal point");
  if (code) return fail(SBFWI_ESINGULAR, "a pivot block of the radial condensation or a separator block of the global matrix is singular");
  return SBFWI_OK;
}

// The exact discrete adjoint's operators for a model set up with the radial finite
// differences: the element set-up runs once more (same density, so mats, rt and S are
// rewritten with the same values) and also emits G_i, rho_0, W, the ghost operators and
// the quadrature factors; the global factors are transposed.
int prepare_exact(Model& md, cudaStream_t st) {
  if (md.exact_ready) return SBFWI_OK;
  if (md.lfe) return fail(SBFWI_EUNSUPPORTED, "the exact adjoint is built for the radial finite differences, not the comparison method");
  const Mesh& m = *md.mesh;
  const int nb = m.nb, n = m.n, L = m.L, ng = (3 * m.p + 2) / 2;
  const int64_t E = m.n_elem, nn = (int64_t)nb * nb;
  SBFWI_CUDA(md.xops.alloc(sizeof(double) * E * n * nn));
  SBFWI_CUDA(md.xel.alloc(sizeof(double) * E * 6 * nn));
  SBFWI_CUDA(md.kq.alloc(sizeof(double) * E * L * ng * 4));
  SBFWI_CUDA(cudaMemsetAsync(md.xops.p, 0, md.xops.bytes, st));
  SBFWI_CUDA(cudaMemsetAsync(md.xel.p, 0, md.xel.bytes, st));
  SBFWI_CUDA(cudaMemsetAsync(md.kq.p, 0, md.kq.bytes, st));
  DevBuf status;
  SBFWI_CUDA(status.alloc(sizeof(int)));
  SBFWI_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st));
  Profiler& prof = profiler();
  prof.begin(kPhaseSetup, st);
  int rc = launch_element_setup(md, m, md.rho_nodal.as<double>(), md.rho_lo.as<double>(), nullptr, md.xops.as<double>(),
                                md.xel.as<double>(), md.kq.as<double>(), status.as<int>(), st);
  if (rc) return rc;
  const Tree& t = m.tree;
  SBFWI_CUDA(md.factors_t.alloc(sizeof(double) * (size_t)std::max<int64_t>(t.X_total, 1)));
  const int tn = (int)t.nodes.size();
  transpose_factors_kernel<<<(unsigned)std::min(tn, 152 * 8), 256, 0, st>>>(m.dev->tree_nodes.as<TreeNodeDev>(), tn,
                                                                           md.factors.as<double>(),
                                                                           md.factors_t.as<double>());
  prof.count(kPhaseSetup);
  SBFWI_CUDA(cudaGetLastError());
  prof.end(kPhaseSetup, st);
  int code = 0;
  if ((rc = read_status(status, st, &code))) return rc;
  if (code) return fail(SBFWI_ESINGULAR, "a pivot block of the radial condensation is singular");
  if (!m.dev->inc_ready) {
    // the elements at each global node (padding dofs, which point at node N, left out)
    std::vector<int64_t> ptr(m.n_nodes + 1, 0), list;
    for (int64_t e = 0; e < E; ++e)
      for (int j = 0; j < m.nbe[e]; ++j) ++ptr[m.dofs[e * nb + j] + 1];
    for (int64_t g = 0; g < m.n_nodes; ++g) ptr[g + 1] += ptr[g];
    list.resize(ptr[m.n_nodes]);
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int j = 0; j < m.nbe[e]; ++j) list[fill[m.dofs[e * nb + j]]++] = e * nb + j;
    if ((rc = upload(m.dev->inc_ptr, ptr, st))) return rc;
    if ((rc = upload(m.dev->inc_list, list, st))) return rc;
    SBFWI_CUDA(cudaStreamSynchronize(st));
    m.dev->inc_ready = true;
  }
  md.exact_ready = true;
  return SBFWI_OK;
}

}  // namespace sbfwi
