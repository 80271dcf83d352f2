// The exact discrete adjoint ("Mode X"): the derivative of the discrete misfit with respect
// to the nodal densities, by reverse-mode differentiation of the time loop.
//
// Forward step k (Section 3.3) solves A(rho) x_{k+1} = r_k with r_k = -xi_i^2 M0_i v_k + f_k,
// v_k the Newmark predictor (Eq. (ODE_Newmark)), x_{k+1} = every element's u_{-1}..u_{n+1}
// and the shared boundary u_n; the state is advanced by Eq. (Newmark) and the misfit
// E = 1/2 dt sum (d - u)^2 (Eq. (misfit)) reads the receivers.  The adjoint runs the steps
// backwards.  For step k, with x_bar the adjoint of u_{k+1} (misfit, Newmark update and the
// next step's predictor), mu = A^{-T} x_bar is found with the condensation's own operators
// in reverse (the transposes of the forward sweep, the global solve and the
// back-substitution, in reverse order):
//   up sweep     s_0 = x_bar_0, s_i = x_bar_i - H_{i-1}^T s_{i-1}, element part of the
//                boundary right-hand side -H_{n-1}^T s_{n-1};
//   global       F_bar = A_g^{-T} (x_bar_b + sum_e Z_e^T (-H_{n-1}^T s_{n-1})) = mu_{n+1}
//                (the flux-balance rows), with the transposed multifrontal factors;
//   down sweep   mu_n = -W^T mu_{n+1}, q_{n-1} = s_{n-1} + R^T mu_{n+1},
//                mu_i = G_i^T q_i, v_bar_i = -P_i^T q_i, q_{i-1} = s_{i-1} - Q_i^T q_i,
//                mu_{-1} = -rho_0^T mu_0, v_bar_n(e) = T^T mu_{n+1};
// the predictor's adjoint v_bar flows into the adjoints of u_k, u'_k, u''_k.
// The gradient is dE/drho = -sum_k mu_k^T dR/drho with R the residual of every row
// (rows 0..n: theta u_{i-1} + phi u_i + psi u_{i+1} + xi_i^2 M0_i v_i; rows -1 and n+1:
// the boundary-condition rows).  Every block is a combination of E0, E1, E2, M0 at one
// radial point and of the radial differences of E0, E1 (central inside, one-sided at the
// ends), and these are linear in the densities of the point: E0 = sum_j rho_j E0hat_j with
// E0hat_j = int phi_j c^2 (b1.b1) phi^T phi det J_b d eta (Eq. (Es)).  So each row's share
// is a sum of Gauss-point products of the interpolated mu and u fields (and their eta
// derivatives), accumulated per radial point, line element and Gauss point over the time
// loop and projected onto phi_j once at the end.
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace sbfwi {

// ---------------------------------------------------------------------------
// element kernel: down sweep of step k fused with the up sweep of step k-1
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) exact_element_kernel(ExactElemArgs a) {
  extern __shared__ double sh[];
  const int nb = a.nb, n = a.n, B = a.B;
  const int per = nb * B;
  const int tid = threadIdx.x;
  const int le = tid / per, rem = tid - le * per, r = rem / B, s = rem - r * B;
  const int64_t e = (int64_t)blockIdx.x * a.epc + le;
  const bool act = (le < a.epc) && (e < a.E);
  double* tbuf = sh + (size_t)le * n * per;                                  // [n][nb][B]
  double* xb = sh + (size_t)a.epc * n * per + (size_t)le * 4 * per;         // four exchange vectors
  double* xc = xb + per;
  double* xd = xc + per;
  double* xe = xd + per;
  const int64_t nn = (int64_t)nb * nb;
  const int64_t ee = act ? e : 0;
  const double* Me = a.mats + ee * (int64_t)n * 3 * nn;
  const double* Ge = a.xops + ee * (int64_t)n * nn;
  const double* Xe = a.xel + ee * 6 * nn;
  const double* RT = a.rt + ee * 2 * nn;
  const int64_t base = ee * (int64_t)n * per;
  const int64_t mrow = ee * (int64_t)(n + 2) * per;                           // mu rows -1..n of this element
  const int rs = r * B + s;
  const int32_t gnode = act ? a.dofs[ee * nb + r] : 0;
  const bool real_node = act && gnode < a.N;                                  // padding dofs point at node N

  if (a.do_down) {
    xb[rs] = real_node ? a.fbar[(int64_t)gnode * B + s] : 0.0;               // mu_{n+1}
    __syncthreads();
    double qv = 0.0, mu0 = 0.0;
    if (act) {
      const double* W = Xe + nn;
      const double* T = RT + nn;
      double aw = 0.0, at = 0.0, ar = 0.0;
      for (int c = 0; c < nb; ++c) {
        const double x = xb[c * B + s];
        aw = fma(W[c * nb + r], x, aw);
        at = fma(T[c * nb + r], x, at);
        ar = fma(RT[c * nb + r], x, ar);
      }
      a.mu[mrow + (int64_t)(n + 1) * per + rs] = -aw;                        // mu_n
      a.vbn[(ee * nb + r) * B + s] = at;                                      // v_bar_n of this element
      qv = a.s[base + (int64_t)(n - 1) * per + rs] + ar;
    }
    __syncthreads();
    xb[rs] = qv;
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {
      double qn = 0.0;
      if (act) {
        const double* G = Ge + (int64_t)i * nn;
        const double* P = Me + (int64_t)i * 3 * nn;
        const double* Q = P + nn;
        double ag = 0.0, ap = 0.0, aq = 0.0;
        for (int c = 0; c < nb; ++c) {
          const double x = xb[c * B + s];
          ag = fma(G[c * nb + r], x, ag);
          ap = fma(P[c * nb + r], x, ap);
          aq = fma(Q[c * nb + r], x, aq);
        }
        a.mu[mrow + (int64_t)(i + 1) * per + rs] = ag;
        if (i == 0) mu0 = ag;
        const double vbar = -ap;
        // Newmark: adjoints of u, u', u'' at step k from those at k+1 and the predictor's
        const int64_t o = base + (int64_t)i * per + rs;
        const double ud1 = a.uda[o], udd1 = a.udda[o];
        const double uk = fma(a.a0, vbar, fma(-a.cu, ud1, -a.du * udd1));
        const double udk = fma(a.a1, vbar, fma(a.cud, ud1, a.dud * udd1));
        const double uddk = fma(a.a2, vbar, fma(a.cudd, ud1, a.dudd * udd1));
        a.ua[o] = uk; a.uda[o] = udk; a.udda[o] = uddk;
        tbuf[(int64_t)i * per + rs] = fma(a.cu, udk, fma(a.du, uddk, uk));  // x_bar_i of step k-1
        if (i > 0) qn = a.s[base + (int64_t)(i - 1) * per + rs] - aq;
      }
      __syncthreads();
      xb[rs] = qn;
      __syncthreads();
    }
    // mu_{-1} = -rho_0^T mu_0
    xb[rs] = mu0;
    __syncthreads();
    if (act) {
      double acc = 0.0;
      for (int c = 0; c < nb; ++c) acc = fma(Xe[c * nb + r], xb[c * B + s], acc);
      a.mu[mrow + rs] = -acc;
    }
    // ghosts of the forward solution x_{k+1}: u_{-1} = u_1 + Gamma u_0,
    // u_{n+1} = -(Y_theta u_{n-1} + Y_phi u_n - Y_M u''_n)
    __syncthreads();
    if (act) {
      const int64_t fb = ee * (int64_t)n * per + rs;
      xb[rs] = a.fu_int[fb];                                                  // u_0
      xc[rs] = a.fu_int[fb + (int64_t)(n - 1) * per];                         // u_{n-1}
      xd[rs] = real_node ? a.fu_b[(int64_t)gnode * B + s] : 0.0;              // u_n
      xe[rs] = real_node ? a.fa_b[(int64_t)gnode * B + s] : 0.0;              // u''_n
    }
    __syncthreads();
    if (act) {
      const double* Gam = Xe + 2 * nn + (int64_t)r * nb;
      const double* Yt = Xe + 3 * nn + (int64_t)r * nb;
      const double* Yp = Xe + 4 * nn + (int64_t)r * nb;
      const double* Ym = Xe + 5 * nn + (int64_t)r * nb;
      double g0 = a.fu_int[ee * (int64_t)n * per + (int64_t)(n > 1 ? 1 : 0) * per + rs];   // u_1 (n >= 2)
      double g1 = 0.0;
      for (int c = 0; c < nb; ++c) {
        const int cs = c * B + s;
        g0 = fma(Gam[c], xb[cs], g0);
        g1 = fma(Yt[c], xc[cs], g1);
        g1 = fma(Yp[c], xd[cs], g1);
        g1 = fma(-Ym[c], xe[cs], g1);
      }
      a.ghost[(ee * 2) * per + rs] = g0;
      a.ghost[(ee * 2 + 1) * per + rs] = -g1;
    }
  } else if (a.do_up && act) {
    for (int i = 0; i < n; ++i) {
      const int64_t o = base + (int64_t)i * per + rs;
      tbuf[(int64_t)i * per + rs] = fma(a.cu, a.uda[o], fma(a.du, a.udda[o], a.ua[o]));
    }
  }
  if (!a.do_up) return;
  __syncthreads();
  // up sweep of step k-1: s_0 = x_bar_0, s_i = x_bar_i - H_{i-1}^T s_{i-1}
  for (int i = 0; i < n; ++i) {
    double v = 0.0;
    if (act) {
      v = tbuf[(int64_t)i * per + rs];
      if (i > 0) {
        const double* H = Me + (int64_t)(i - 1) * 3 * nn + 2 * nn;
        for (int c = 0; c < nb; ++c) v = fma(-H[c * nb + r], xb[c * B + s], v);
      }
      a.s[base + (int64_t)i * per + rs] = v;
    }
    __syncthreads();
    xb[rs] = v;
    __syncthreads();
  }
  if (act) {
    const double* H = Me + (int64_t)(n - 1) * 3 * nn + 2 * nn;
    double acc = 0.0;
    for (int c = 0; c < nb; ++c) acc = fma(H[c * nb + r], xb[c * B + s], acc);
    a.fhat[(ee * nb + r) * B + s] = -acc;
  }
}

// ---------------------------------------------------------------------------
// boundary nodes
// ---------------------------------------------------------------------------
// the misfit's share: the adjoint of u at the receivers after step k gets -dt (d - u)
__global__ void exact_misfit_kernel(double* ub, int B, int R, const int64_t* rec, const double* res, int64_t K,
                                    int64_t k, double dt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * R) return;
  const int s = t / R, j = t - s * R;
  ub[rec[j] * B + s] -= dt * res[((int64_t)s * R + j) * K + k];
}

// x_bar of the boundary nodes for the transposed solve, and the Newmark update's share of
// the adjoints of u, u', u'' at step k
__global__ void exact_boundary_pre_kernel(ExactBoundaryArgs a) {
  const int64_t tot = a.N * a.B;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const double u1 = a.ub[t], ud1 = a.udb[t], udd1 = a.uddb[t];
    a.ext[t] = fma(a.cu, ud1, fma(a.du, udd1, u1));
    a.ub[t] = fma(-a.cu, ud1, -a.du * udd1);
    a.udb[t] = fma(a.cud, ud1, a.dud * udd1);
    a.uddb[t] = fma(a.cudd, ud1, a.dudd * udd1);
  }
}

// the predictor's share: v_bar of a node is the sum of its elements' T^T mu_{n+1}
__global__ void exact_boundary_post_kernel(ExactBoundaryArgs a) {
  const int64_t tot = a.N * a.B;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = t / a.B;
    const int s = (int)(t - g * a.B);
    double v = 0.0;
    for (int64_t l = a.inc_ptr[g]; l < a.inc_ptr[g + 1]; ++l) v += a.vbn[a.inc_list[l] * a.B + s];
    a.ub[t] = fma(a.a0, v, a.ub[t]);
    a.udb[t] = fma(a.a1, v, a.udb[t]);
    a.uddb[t] = fma(a.a2, v, a.uddb[t]);
  }
}

// ---------------------------------------------------------------------------
// gradient: Gauss-point products of one step
// ---------------------------------------------------------------------------
struct Acc4 {
  double e0, e1, e2, m;
};
__device__ __forceinline__ void zero4(Acc4& x) { x.e0 = x.e1 = x.e2 = x.m = 0.0; }

// sum over the Bp lanes of one (element, line, Gauss point), then one lane adds the station's
// four sums to the accumulators
__device__ __forceinline__ void flush4(const ExactGradArgs& a, Acc4 v, int64_t e, int st, int l, int g, int lane,
                                       int Bp, bool live) {
  for (int off = Bp >> 1; off > 0; off >>= 1) {
    v.e0 += __shfl_xor_sync(0xffffffffu, v.e0, off);
    v.e1 += __shfl_xor_sync(0xffffffffu, v.e1, off);
    v.e2 += __shfl_xor_sync(0xffffffffu, v.e2, off);
    v.m += __shfl_xor_sync(0xffffffffu, v.m, off);
  }
  if (live && lane == 0) {
    const int64_t LG = (int64_t)a.L * a.ng;
    double* acc = a.gacc + ((e * (a.n + 1) + st) * 4) * LG + (int64_t)l * a.ng + g;
    acc[0] += v.e0;
    acc[LG] += v.e1;
    acc[2 * LG] += v.e2;
    acc[3 * LG] += v.m;
  }
}

template <int PP>
__global__ void __launch_bounds__(256) exact_gradient_kernel(ExactGradArgs a) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int Bp = a.Bp;
  const int lane = (int)(t % Bp);
  const int64_t grp = t / Bp;                      // (e, line, Gauss point)
  const int ng = a.ng;
  const int g = (int)(grp % ng);
  const int64_t el = grp / ng;
  const int l = (int)(el % a.L);
  const int64_t e = el / a.L;
  const bool in_range = e < a.E;
  const int64_t ee = in_range ? e : 0;
  const int L_e = (int)(a.lptr[ee + 1] - a.lptr[ee]);
  // a whole warp takes part in the shuffles: lanes outside the problem compute zeros
  const bool live = in_range && l < L_e;
  const int s = lane < a.B ? lane : 0;
  const bool shot = live && lane < a.B;
  const int nb = a.nb, n = a.n, B = a.B;
  const int per = nb * B;
  double ph[PP], dph[PP];
  int loc[PP];
#pragma unroll
  for (int q = 0; q < PP; ++q) {
    ph[q] = a.tab[2 * (ng + g * PP + q)];
    dph[q] = a.tab[2 * (ng + ng * PP + g * PP + q)];
    loc[q] = live ? a.line_local[(a.lptr[ee] + l) * PP + q] : 0;
  }
  const double h = a.h;
  const double* fu_int = a.fu_int + ee * (int64_t)n * per;
  const double* fa_int = a.fa_int + ee * (int64_t)n * per;
  const double* mu = a.mu + ee * (int64_t)(n + 2) * per;
  const double* gh = a.ghost + ee * 2 * per;
  const int32_t* dofs = a.dofs + ee * nb;
  // value and eta-derivative at this Gauss point of a field row given per local dof
  auto interp_row = [&](const double* row, double& v, double& d) {
    v = 0.0; d = 0.0;
#pragma unroll
    for (int q = 0; q < PP; ++q) {
      const double x = shot ? row[loc[q] * B + s] : 0.0;
      v = fma(ph[q], x, v);
      d = fma(dph[q], x, d);
    }
  };
  auto interp_nodes = [&](const double* glob, double& v, double& d) {   // a row on the global nodes
    v = 0.0; d = 0.0;
#pragma unroll
    for (int q = 0; q < PP; ++q) {
      const int32_t gn = dofs[loc[q]];
      const double x = (shot && gn < a.N) ? glob[(int64_t)gn * B + s] : 0.0;
      v = fma(ph[q], x, v);
      d = fma(dph[q], x, d);
    }
  };
  // the forward solution's row r = -1..n+1 (ghosts, interior, boundary nodes)
  auto u_row = [&](int r, double& v, double& d) {
    if (r == -1) interp_row(gh, v, d);
    else if (r < n) interp_row(fu_int + (int64_t)r * per, v, d);
    else if (r == n) interp_nodes(a.fu_b, v, d);
    else interp_row(gh + per, v, d);
  };
  double uA, uAd, uB, uBd, uC, uCd, mv, md, av, ad;
  Acc4 prv, cur, nxt;
  zero4(prv); zero4(cur); zero4(nxt);
  u_row(-1, uA, uAd);
  u_row(0, uB, uBd);
  u_row(1, uC, uCd);
  const double inv_2h = 0.5 / h;
  // row -1 (station 0): xi_0 E0_0 (u_1 - u_{-1}) / (2h) + E1_0^T u_0
  interp_row(mu, mv, md);
  {
    const double x0 = a.xi[0];
    cur.e0 = fma(x0 * inv_2h * mv, uC - uA, cur.e0);
    cur.e1 = fma(uBd, mv, cur.e1);
  }
  for (int r = 0; r <= n; ++r) {
    if (r > 0) {
      uA = uB; uAd = uBd; uB = uC; uBd = uCd;
      u_row(r + 1, uC, uCd);
    }
    interp_row(mu + (int64_t)(r + 1) * per, mv, md);
    if (r < n) interp_row(fa_int + (int64_t)r * per, av, ad);
    else interp_nodes(a.fa_b, av, ad);
    const double xi = a.xi[r];
    const double d1 = uC - uA, d1d = uCd - uAd, d2 = uA - 2.0 * uB + uC;
    cur.e0 = fma(mv, fma(xi * xi / (h * h), d2, xi * inv_2h * d1), cur.e0);
    cur.e1 = fma(xi * inv_2h, fma(d1d, mv, -md * d1), cur.e1);
    cur.e2 = fma(-md, uBd, cur.e2);
    cur.m = fma(-xi * xi * mv, av, cur.m);
    // radial differences of E0 and E1: forward at r = 0, backward at r = n, central inside
    const double te0 = xi * xi * inv_2h * mv * d1;     // times the weight of E0 at a station
    const double te1 = xi * uBd * mv;                  // times the weight of E1 at a station
    if (r == 0) {
      const double w = 1.0 / h;
      nxt.e0 = fma(w, te0, nxt.e0); nxt.e1 = fma(w, te1, nxt.e1);
      cur.e0 = fma(-w, te0, cur.e0); cur.e1 = fma(-w, te1, cur.e1);
    } else if (r == n) {
      const double w = 1.0 / h;
      cur.e0 = fma(w, te0, cur.e0); cur.e1 = fma(w, te1, cur.e1);
      prv.e0 = fma(-w, te0, prv.e0); prv.e1 = fma(-w, te1, prv.e1);
    } else {
      nxt.e0 = fma(inv_2h, te0, nxt.e0); nxt.e1 = fma(inv_2h, te1, nxt.e1);
      prv.e0 = fma(-inv_2h, te0, prv.e0); prv.e1 = fma(-inv_2h, te1, prv.e1);
    }
    if (r == n) break;
    // station r - 1 is complete
    if (r >= 1) flush4(a, prv, ee, r - 1, l, g, lane, Bp, live);
    prv = cur; cur = nxt; zero4(nxt);
  }
  // row n+1 (station n): xi_n E0_n (u_{n+1} - u_{n-1}) / (2h) + E1_n^T u_n, mu_{n+1} on the global nodes
  interp_nodes(a.fbar, mv, md);
  {
    const double xn = a.xi[n];
    cur.e0 = fma(xn * inv_2h * mv, uC - uA, cur.e0);
    cur.e1 = fma(uBd, mv, cur.e1);
  }
  flush4(a, prv, ee, n - 1, l, g, lane, Bp, live);
  flush4(a, cur, ee, n, l, g, lane, Bp, live);
}

// dE/drho at every radial point and boundary node of every element from the accumulated
// products: -sum_lines sum_g phi_j(g) (k0 A0 + k1 A1 + k2 A2 + km Am); interior points go to
// the library's nodal layout, the boundary station to a per-element slot (gathered per node)
__global__ void exact_finalize_kernel(ExactFinalArgs a) {
  const int nb = a.nb, n = a.n, pp = a.pp, ng = a.ng;
  const int64_t tot = a.E * (int64_t)(n + 1) * nb;
  const int64_t LG = (int64_t)a.L * ng;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / ((int64_t)(n + 1) * nb);
    const int rem = (int)(t - e * (int64_t)(n + 1) * nb);
    const int st = rem / nb, j = rem - st * nb;
    const int64_t l0 = a.lptr[e];
    const int Le = (int)(a.lptr[e + 1] - l0);
    const double* acc = a.gacc + ((e * (n + 1) + st) * 4) * LG;
    double sum = 0.0;
    for (int l = 0; l < Le; ++l) {
      for (int q = 0; q < pp; ++q) {
        if (a.line_local[(l0 + l) * pp + q] != j) continue;
        for (int g = 0; g < ng; ++g) {
          const double* k = a.kq + ((e * a.L + l) * ng + g) * 4;
          const int64_t o = (int64_t)l * ng + g;
          const double v = k[0] * acc[o] + k[1] * acc[LG + o] + k[2] * acc[2 * LG + o] + k[3] * acc[3 * LG + o];
          sum = fma(a.tab[2 * (ng + g * pp + q)], v, sum);
        }
      }
    }
    if (st < n) a.g_nodal[(e * n + st) * nb + j] = -sum;
    else a.g_bnd[e * nb + j] = -sum;
  }
}

__global__ void exact_gather_nodes_kernel(const double* g_bnd, const int64_t* inc_ptr, const int64_t* inc_list,
                                          int64_t N, double* g_nodal_b) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int64_t l = inc_ptr[g]; l < inc_ptr[g + 1]; ++l) v += g_bnd[inc_list[l]];
    g_nodal_b[g] = v;
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int exact_element_launch(const ExactElemArgs& a, cudaStream_t st) {
  const int threads = a.epc * a.nb * a.B;
  const unsigned blocks = (unsigned)((a.E + a.epc - 1) / a.epc);
  const size_t smem = exact_element_smem(a.nb, a.n, a.B, a.epc);
  if (smem > 48 * 1024)
    SBFWI_CUDA(cudaFuncSetAttribute(exact_element_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  exact_element_kernel<<<blocks, threads, smem, st>>>(a);
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

size_t exact_element_smem(int nb, int n, int B, int epc) {
  return sizeof(double) * (size_t)epc * (n + 4) * nb * B;
}

int exact_misfit_launch(double* ub, int B, int R, const int64_t* rec, const double* res, int64_t K, int64_t k, double dt,
                        cudaStream_t st) {
  if (R == 0) return SBFWI_OK;
  exact_misfit_kernel<<<(B * R + 127) / 128, 128, 0, st>>>(ub, B, R, rec, res, K, k, dt);
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

int exact_boundary_launch(const ExactBoundaryArgs& a, bool post, cudaStream_t st) {
  const unsigned blocks = (unsigned)std::min<int64_t>((a.N * a.B + 255) / 256, 152 * 8);
  if (post) exact_boundary_post_kernel<<<blocks, 256, 0, st>>>(a);
  else exact_boundary_pre_kernel<<<blocks, 256, 0, st>>>(a);
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

int exact_gradient_launch(const ExactGradArgs& a, int p, cudaStream_t st) {
  const int64_t threads = a.E * (int64_t)a.L * a.ng * a.Bp;
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  switch (p + 1) {
    case 2: exact_gradient_kernel<2><<<blocks, 256, 0, st>>>(a); break;
    case 3: exact_gradient_kernel<3><<<blocks, 256, 0, st>>>(a); break;
    case 4: exact_gradient_kernel<4><<<blocks, 256, 0, st>>>(a); break;
    case 5: exact_gradient_kernel<5><<<blocks, 256, 0, st>>>(a); break;
    case 6: exact_gradient_kernel<6><<<blocks, 256, 0, st>>>(a); break;
    case 7: exact_gradient_kernel<7><<<blocks, 256, 0, st>>>(a); break;
    case 8: exact_gradient_kernel<8><<<blocks, 256, 0, st>>>(a); break;
    case 9: exact_gradient_kernel<9><<<blocks, 256, 0, st>>>(a); break;
    default: return fail(SBFWI_EUNSUPPORTED, "line order outside 1..8");
  }
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

int exact_finalize_launch(const ExactFinalArgs& a, const int64_t* inc_ptr, const int64_t* inc_list, int64_t N,
                          double* g_nodal_b, cudaStream_t st) {
  const int64_t tot = a.E * (int64_t)(a.n + 1) * a.nb;
  exact_finalize_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16), 256, 0, st>>>(a);
  exact_gather_nodes_kernel<<<(unsigned)std::min<int64_t>((N + 255) / 256, 152 * 8), 256, 0, st>>>(
      a.g_bnd, inc_ptr, inc_list, N, g_nodal_b);
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

}  // namespace sbfwi
