// The time loop of the path: forward and time-reversed adjoint solves, the
// zero-lag cross-correlation kernel, the misfit, and the C-ABI entry points.
//
// One Newmark step (Section 3.3; Eq. (Newmark), Eq. (ODE_Newmark)) of every
// element and shot is split into
//   A  forward sweep:  q_i = -(P_i v_i + Q_i q_{i-1}),  i = 0..n-1,
//                      f_hat = R q_{n-1} + T v_n,
//      with v the Newmark predictor u/(beta dt^2) + u'/(beta dt) + (1/(2 beta) - 1) u''
//      and q_i = phi_i^{-1} p_i the pivot-normalised right-hand side of the
//      paper's Thomas sweep (p_i -= varrho_i p_{i-1} with varrho_i = theta_i phi_{i-1}^{-1});
//   B  global boundary solve of sum_e S_e u_n = sum_e f_hat_e + f along the
//      elimination tree (forward pass leaves -> root, backward pass root -> leaves),
//      then the Newmark update of the boundary nodes, receivers and the forward
//      store / the gradient at the boundary nodes;
//   C  back-substitution u_i = q_i - H_i u_{i+1} (= phi_i^{-1}(p_i - psi_i u_{i+1})),
//      i = n-1..0, Newmark update of the interior, forward store / gradient.
// Kernel E fuses C of step k with A of step k+1 (the back-substitution runs from
// the boundary inwards, the next forward sweep from the centre outwards), so the
// interior state is read and written once per step.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "internal.h"
#include "sync.cuh"
#include "prof.h"

namespace sbfwi {

int setup_model(Model& md, const Mesh& m, const double* rho, int mem, cudaStream_t st);

static constexpr int kMaxShots = 16;

// ---------------------------------------------------------------------------
// kernel E: back-substitution + Newmark (step k) fused with the forward sweep (step k+1)
// ---------------------------------------------------------------------------
struct ElemStepArgs {
  int nb, n, B, epc;
  int64_t E;
  double a0, a1, a2, c1, c2, dt;
  const double* mats;   // [E][n][3][nb][nb] P, Q, H
  const double* rt;     // [E][2][nb][nb]    R, T
  const int32_t* dofs;  // [E][nb]
  double* u; double* ud; double* udd;            // interior state [E][n][nb][B]
  const double* ub; const double* udb; const double* uddb;  // boundary state [N][B]
  double* q;            // [E][n][nb][B]
  double* fhat;         // [E][nb][B]
  int do_down, do_up;
  double* store_int;    // forward: velocities of this step, interior part [E][n][nb][B]
  const double* fwd_int;// adjoint: paired forward velocities, interior part
  double* grad_int;     // adjoint: accumulators [E][n][nb][B]
  double* u_out;        // full Frechet kernel, exact adjoint: the new interior displacements [E][n][nb][B]
  double* a_out;        // exact adjoint: the new interior accelerations [E][n][nb][B]
  const int32_t* elems; // the elements of this launch (an element class), or NULL for all
  int64_t n_elems;
};

__global__ void __launch_bounds__(512) element_step_kernel(ElemStepArgs a) {
  extern __shared__ double sh[];
  const int nb = a.nb, n = a.n, B = a.B;
  const int per = nb * B;
  const int tid = threadIdx.x;
  const int le = tid / per, rem = tid - le * per, r = rem / B, s = rem - r * B;
  const int64_t idx = (int64_t)blockIdx.x * a.epc + le;
  const bool act = (le < a.epc) && (idx < a.n_elems);
  const int64_t e = act ? (a.elems ? (int64_t)a.elems[idx] : idx) : 0;
  double* vbuf = sh + (size_t)le * n * per;                 // [n][nb][B] predictors of the new state
  double* xb = sh + (size_t)a.epc * n * per + (size_t)le * per;   // [nb][B] exchange
  double* vn = sh + (size_t)a.epc * (n + 1) * per + (size_t)le * per;
  const int64_t nn = (int64_t)nb * nb;
  const double* Me = a.mats + (act ? e : 0) * (int64_t)n * 3 * nn;
  const int64_t base = (act ? e : 0) * (int64_t)n * per;    // interior offset of this element

  if (a.do_down) {
    if (act) xb[r * B + s] = a.ub[(int64_t)a.dofs[e * nb + r] * B + s];
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {
      double un = 0.0;
      if (act) {
        const int64_t o = base + (int64_t)i * per + r * B + s;
        const double* H = Me + (int64_t)i * 3 * nn + 2 * nn + (int64_t)r * nb;
        double acc = a.q[o];
        for (int c = 0; c < nb; ++c) acc = fma(-H[c], xb[c * B + s], acc);
        un = acc;
        const double uo = a.u[o], udo = a.ud[o], uddo = a.udd[o];
        const double vo = fma(a.a0, uo, fma(a.a1, udo, a.a2 * uddo));
        const double uddn = fma(a.a0, un, -vo);
        const double udn = fma(a.c2, uddn, fma(a.c1, uddo, udo));
        a.u[o] = un; a.ud[o] = udn; a.udd[o] = uddn;
        if (a.store_int) a.store_int[o] = udn;
        if (a.grad_int) a.grad_int[o] = fma(a.fwd_int[o], udn, a.grad_int[o]);   // dt applied at the end
        if (a.u_out) a.u_out[o] = un;
        if (a.a_out) a.a_out[o] = uddn;
        if (a.do_up) vbuf[i * per + r * B + s] = fma(a.a0, un, fma(a.a1, udn, a.a2 * uddn));
      }
      __syncthreads();
      if (act) xb[r * B + s] = un;
      __syncthreads();
    }
  } else if (a.do_up && act) {
    for (int i = 0; i < n; ++i) {
      const int64_t o = base + (int64_t)i * per + r * B + s;
      vbuf[i * per + r * B + s] = fma(a.a0, a.u[o], fma(a.a1, a.ud[o], a.a2 * a.udd[o]));
    }
  }
  if (!a.do_up) return;
  if (act) {
    const int64_t g = (int64_t)a.dofs[e * nb + r] * B + s;
    vn[r * B + s] = fma(a.a0, a.ub[g], fma(a.a1, a.udb[g], a.a2 * a.uddb[g]));
  }
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    double qv = 0.0;
    if (act) {
      const double* P = Me + (int64_t)i * 3 * nn + (int64_t)r * nb;
      const double* v = vbuf + i * per;
      double acc = 0.0;
      for (int c = 0; c < nb; ++c) acc = fma(P[c], v[c * B + s], acc);
      if (i > 0) {
        const double* Q = P + nn;
        for (int c = 0; c < nb; ++c) acc = fma(Q[c], xb[c * B + s], acc);
      }
      qv = -acc;
      a.q[base + (int64_t)i * per + r * B + s] = qv;
    }
    __syncthreads();
    if (act) xb[r * B + s] = qv;
    __syncthreads();
  }
  if (act) {
    const double* R = a.rt + e * 2 * nn + (int64_t)r * nb;
    const double* T = R + nn;
    double acc = 0.0;
    for (int c = 0; c < nb; ++c) acc = fma(R[c], xb[c * B + s], acc);
    for (int c = 0; c < nb; ++c) acc = fma(T[c], vn[c * B + s], acc);
    a.fhat[(e * nb + r) * B + s] = acc;
  }
}

// ---------------------------------------------------------------------------
// kernel B: global boundary solve, one launch per tree level and direction
// ---------------------------------------------------------------------------
struct SolveArgs {
  const int32_t* sep_nodes;
  const int32_t* bnd_nodes;
  const int32_t* src0;   // per front position: row of ybnd (or f_hat in a leaf); <= -2: f_hat row -2 - v
                         // of a pass-through child leaf; -1 absent
  const int32_t* src1;
  const double* factors;
  const double* fhat;    // [E][nb][B]
  const double* ext;     // [N][B] external sources
  double* ysep;          // [sep_rows][B]
  double* ybnd;          // [bnd_rows][B]
  double* x;             // [N][B] solution
  int nb, B;
  unsigned bdiv;         // floor(2^32 / B) + 1 (B >= 2): see div_shots
  int warp_doubles;      // shared memory of one warp task (doubles)
};

// Sources of a front position: rows of f_hat (r <= -2: the leaf's own element, or a
// pass-through child leaf) and the external sources are written before the solve
// starts; rows of ybnd (r >= 0, a child's boundary) are written by other tasks of the
// same solve (read through L2).  r = -1: absent.  Staging reads the first kind before
// a task waits for its inputs and only the second kind after the wait.
__device__ __forceinline__ double fhat_part(const SolveArgs& a, int32_t r, int s) {
  return r <= -2 ? __ldcg(a.fhat + (int64_t)(-2 - r) * a.B + s) : 0.0;
}
__device__ __forceinline__ double ybnd_part(const SolveArgs& a, int32_t r, int s) {
  return r >= 0 ? __ldcg(a.ybnd + (int64_t)r * a.B + s) : 0.0;
}

// t / B for 0 <= t < 2^20: a multiply by floor(2^32 / B) + 1 and the high word (exact in
// that range for B < 4096), instead of an integer division
__device__ __forceinline__ int div_shots(const SolveArgs& a, int t) {
  return a.B == 1 ? t : (int)__umulhi((unsigned)t, a.bdiv);
}

// sum over the ks consecutive lanes that share one output (ks in {1, 2, ..., 32})
__device__ __forceinline__ double lane_group_sum(double v, int ks) {
  for (int off = ks >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Shared-memory staging of a task, U values per thread at a time: all loads of a batch
// are issued before any of its stores, so the loads of different positions overlap.
// Every task stages in parts: the constant part (factor rows, index arrays, and the
// front values that do not come from other tasks) can be loaded before the task waits
// for its inputs; the data part after.  The data part reads index arrays that the
// constant part wrote, so the two are separated by a block (or warp) barrier.
//
// Forward task (rows r0..r1 of the node's boundary):
//   [front values: c_sep (s B), then c_bnd of the task's rows (rows B) | the task's rows
//    of C (rows x s) | ybnd source rows of those s + rows positions (2 (s + rows) int32)]
// c = ext + f_hat parts + ybnd parts, in this order for every schedule.
struct FwdStage {
  double* vals;
  double* C;
  int32_t* i0;
  int32_t* i1;
  int P, rows;
};
__device__ __forceinline__ FwdStage fwd_layout(const Task& tk, double* sm, int B) {
  FwdStage f;
  f.rows = tk.r1 - tk.r0;
  f.P = tk.s + f.rows;
  f.vals = sm;
  f.C = sm + (size_t)f.P * B;
  f.i0 = reinterpret_cast<int32_t*>(f.C + (size_t)f.rows * tk.s);
  f.i1 = f.i0 + f.P;
  return f;
}

template <int U>
__device__ __forceinline__ void fwd_stage_const(const SolveArgs& a, const Task& tk, double* sm, int tid, int nthr) {
  const int B = a.B, S = tk.s;
  const FwdStage f = fwd_layout(tk, sm, B);
  const double* C = a.factors + tk.X_off + (int64_t)S * S + (int64_t)S * tk.b + (int64_t)tk.r0 * S;
  const int nv = f.P * B, n = nv + f.rows * S;
  for (int base = 0; base < n; base += U * nthr) {
    double v[U];
    int32_t q0[U], q1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      v[u] = 0.0;
      q0[u] = -1;
      q1[u] = -1;
      if (t < nv) {
        const int p = div_shots(a, t), sh = t - p * B;
        const int pos = p < S ? p : S + tk.r0 + (p - S);
        q0[u] = a.src0[tk.map_off + pos];
        q1[u] = a.src1[tk.map_off + pos];
        if (p < S) v[u] = __ldcg(a.ext + (int64_t)a.sep_nodes[tk.sep_off + p] * B + sh);
      } else if (t < n) {
        v[u] = C[t - nv];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < nv) {
        const int p = div_shots(a, t), sh = t - p * B;
        v[u] += fhat_part(a, q0[u], sh);
        v[u] += fhat_part(a, q1[u], sh);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < nv) {
        const int p = div_shots(a, t), sh = t - p * B;
        f.vals[t] = v[u];
        if (sh == 0) {
          f.i0[p] = q0[u];
          f.i1[p] = q1[u];
        }
      } else if (t < n) {
        f.C[t - nv] = v[u];
      }
    }
  }
}

// the ybnd parts (children's boundaries); c_sep also goes to ysep if asked
template <int U>
__device__ __forceinline__ void fwd_stage_data(const SolveArgs& a, const Task& tk, double* sm, bool write_ysep, int tid,
                                               int nthr) {
  const int B = a.B, S = tk.s;
  const FwdStage f = fwd_layout(tk, sm, B);
  const int nv = f.P * B;
  for (int base = 0; base < nv; base += U * nthr) {
    double y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      y[u] = 0.0;
      if (t < nv) {
        const int p = div_shots(a, t), sh = t - p * B;
        y[u] = ybnd_part(a, f.i0[p], sh);
        y[u] += ybnd_part(a, f.i1[p], sh);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < nv) {
        const double c = f.vals[t] + y[u];
        f.vals[t] = c;
        if (write_ysep && t < S * B) a.ysep[tk.sep_off * B + t] = c;
      }
    }
  }
}

// Backward task (rows r0..r1 of the node's separator):
//   [y_sep (s B) | x at the node's boundary nodes (b B) | the task's rows of X (rows x s) |
//    the task's rows of G (rows x b) | boundary node ids (b int32) | separator node ids of
//    the task's rows (rows int32)]
// Parts: constant (factor rows, node ids), own (y_sep: this node's forward tasks) and data
// (x at the boundary: the nearest ancestor's backward tasks).
struct BwdStage {
  double* ys;
  double* xb;
  double* X;
  double* G;
  int32_t* bnd;
  int32_t* sep;
  int rows;
};
__device__ __forceinline__ BwdStage bwd_layout(const Task& tk, double* sm, int B) {
  BwdStage g;
  g.rows = tk.r1 - tk.r0;
  g.ys = sm;
  g.xb = sm + (size_t)tk.s * B;
  g.X = g.xb + (size_t)tk.b * B;
  g.G = g.X + (size_t)g.rows * tk.s;
  g.bnd = reinterpret_cast<int32_t*>(g.G + (size_t)g.rows * tk.b);
  g.sep = g.bnd + tk.b;
  return g;
}

template <int U>
__device__ __forceinline__ void bwd_stage_const(const SolveArgs& a, const Task& tk, double* sm, int tid, int nthr) {
  const int S = tk.s, Bn = tk.b;
  const BwdStage g = bwd_layout(tk, sm, a.B);
  const double* X = a.factors + tk.X_off + (int64_t)tk.r0 * S;
  const double* G = a.factors + tk.X_off + (int64_t)S * S + (int64_t)tk.r0 * Bn;
  const int n1 = g.rows * S, n2 = n1 + g.rows * Bn, n3 = n2 + Bn, n4 = n3 + g.rows;
  for (int base = 0; base < n4; base += U * nthr) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      v[u] = 0.0;
      if (t < n1) v[u] = X[t];
      else if (t < n2) v[u] = G[t - n1];
      else if (t < n3) v[u] = __hiloint2double(0, a.bnd_nodes[tk.bnd_off + (t - n2)]);
      else if (t < n4) v[u] = __hiloint2double(0, a.sep_nodes[tk.sep_off + tk.r0 + (t - n3)]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < n1) g.X[t] = v[u];
      else if (t < n2) g.G[t - n1] = v[u];
      else if (t < n3) g.bnd[t - n2] = __double2loint(v[u]);
      else if (t < n4) g.sep[t - n3] = __double2loint(v[u]);
    }
  }
}

template <int U>
__device__ __forceinline__ void bwd_stage_own(const SolveArgs& a, const Task& tk, double* sm, int tid, int nthr) {
  const BwdStage g = bwd_layout(tk, sm, a.B);
  const int n = tk.s * a.B;
  for (int base = 0; base < n; base += U * nthr) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      v[u] = t < n ? __ldcg(a.ysep + tk.sep_off * a.B + t) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < n) g.ys[t] = v[u];
    }
  }
}

template <int U>
__device__ __forceinline__ void bwd_stage_data(const SolveArgs& a, const Task& tk, double* sm, int tid, int nthr) {
  const int B = a.B;
  const BwdStage g = bwd_layout(tk, sm, B);
  const int n = tk.b * B;
  for (int base = 0; base < n; base += U * nthr) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      v[u] = 0.0;
      if (t < n) {
        const int j = div_shots(a, t), sh = t - j * B;
        v[u] = __ldcg(a.x + (int64_t)g.bnd[j] * B + sh);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < n) g.xb[t] = v[u];
    }
  }
}

// Everything at once, for the schedules that have nothing to wait for (barrier, per
// level): the same values in the same order of summation as the parts, so every schedule
// gives the same bits, in one pass of dependent loads (index, then value).
template <int U>
__device__ __forceinline__ void fwd_stage_all(const SolveArgs& a, const Task& tk, double* sm, bool write_ysep, int tid,
                                              int nthr) {
  const int B = a.B, S = tk.s;
  const FwdStage f = fwd_layout(tk, sm, B);
  const double* C = a.factors + tk.X_off + (int64_t)S * S + (int64_t)S * tk.b + (int64_t)tk.r0 * S;
  const int nv = f.P * B, n = nv + f.rows * S;
  for (int base = 0; base < n; base += U * nthr) {
    double v[U], y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      v[u] = 0.0;
      y[u] = 0.0;
      if (t < nv) {
        const int p = div_shots(a, t), sh = t - p * B;
        const int pos = p < S ? p : S + tk.r0 + (p - S);
        const int32_t q0 = a.src0[tk.map_off + pos], q1 = a.src1[tk.map_off + pos];
        if (p < S) v[u] = __ldcg(a.ext + (int64_t)a.sep_nodes[tk.sep_off + p] * B + sh);
        v[u] += fhat_part(a, q0, sh);
        v[u] += fhat_part(a, q1, sh);
        y[u] = ybnd_part(a, q0, sh);
        y[u] += ybnd_part(a, q1, sh);
      } else if (t < n) {
        v[u] = C[t - nv];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < nv) {
        const double c = v[u] + y[u];
        f.vals[t] = c;
        if (write_ysep && t < S * B) a.ysep[tk.sep_off * B + t] = c;
      } else if (t < n) {
        f.C[t - nv] = v[u];
      }
    }
  }
}

template <int U>
__device__ __forceinline__ void bwd_stage_all(const SolveArgs& a, const Task& tk, double* sm, int tid, int nthr) {
  const int B = a.B, S = tk.s, Bn = tk.b;
  const BwdStage g = bwd_layout(tk, sm, B);
  const double* X = a.factors + tk.X_off + (int64_t)tk.r0 * S;
  const double* G = a.factors + tk.X_off + (int64_t)S * S + (int64_t)tk.r0 * Bn;
  const int n1 = S * B, n2 = n1 + Bn * B, n3 = n2 + g.rows * S, n4 = n3 + g.rows * Bn, n5 = n4 + g.rows;
  for (int base = 0; base < n5; base += U * nthr) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      v[u] = 0.0;
      if (t < n1) {
        v[u] = __ldcg(a.ysep + tk.sep_off * B + t);
      } else if (t < n2) {
        const int q = t - n1, j = div_shots(a, q), sh = q - j * B;
        v[u] = __ldcg(a.x + (int64_t)a.bnd_nodes[tk.bnd_off + j] * B + sh);
      } else if (t < n3) {
        v[u] = X[t - n2];
      } else if (t < n4) {
        v[u] = G[t - n3];
      } else if (t < n5) {
        v[u] = __hiloint2double(0, a.sep_nodes[tk.sep_off + tk.r0 + (t - n4)]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = base + u * nthr + tid;
      if (t < n1) g.ys[t] = v[u];
      else if (t < n2) g.xb[t - n1] = v[u];
      else if (t < n3) g.X[t - n2] = v[u];
      else if (t < n4) g.G[t - n3] = v[u];
      else if (t < n5) g.sep[t - n4] = __double2loint(v[u]);
    }
  }
}

// forward products of a block task: y_bnd = c_bnd - C c_sep for the task's rows
__device__ void fwd_compute_block(const SolveArgs& a, const Task& tk, const double* sm) {
  const int B = a.B, S = tk.s;
  const FwdStage f = fwd_layout(tk, const_cast<double*>(sm), B);
  const double* csep = f.vals;
  const double* cb = f.vals + (size_t)S * B;
  const int ks = tk.ksplit, kl = __ffs(ks) - 1;     // ks: a power of two
  const int outputs = f.rows * B;
  // every lane walks the same number of rounds so that the lane-group shuffles see full warps
  const int rounds = (outputs * ks + blockDim.x - 1) / blockDim.x;
  for (int rd = 0; rd < rounds; ++rd) {
    const int t = rd * blockDim.x + threadIdx.x;
    const int o = t >> kl, kk = t & (ks - 1);
    const bool live = o < outputs;
    const int ro = live ? div_shots(a, o) : 0, sh = live ? o - ro * B : 0;
    double acc = 0.0;
    if (live) {
      const double* Cr = f.C + ro * S;
#pragma unroll 4
      for (int k = kk; k < S; k += ks) acc = fma(Cr[k], csep[k * B + sh], acc);
    }
    acc = lane_group_sum(acc, ks);
    if (live && kk == 0) a.ybnd[(tk.bnd_off + tk.r0 + ro) * B + sh] = cb[ro * B + sh] - acc;
  }
}

// backward products of a block task: x_sep = X y_sep - G x_bnd for the task's rows
__device__ void bwd_compute_block(const SolveArgs& a, const Task& tk, const double* sm) {
  const int B = a.B, S = tk.s, Bn = tk.b;
  const BwdStage g = bwd_layout(tk, const_cast<double*>(sm), B);
  const int ks = tk.ksplit, kl = __ffs(ks) - 1;     // ks: a power of two
  const int outputs = g.rows * B;
  const int rounds = (outputs * ks + blockDim.x - 1) / blockDim.x;
  for (int rd = 0; rd < rounds; ++rd) {
    const int t = rd * blockDim.x + threadIdx.x;
    const int o = t >> kl, kk = t & (ks - 1);
    const bool live = o < outputs;
    const int ro = live ? div_shots(a, o) : 0, sh = live ? o - ro * B : 0;
    double acc = 0.0;
    if (live) {
      const double* Xr = g.X + ro * S;
#pragma unroll 4
      for (int k = kk; k < S; k += ks) acc = fma(Xr[k], g.ys[k * B + sh], acc);
      const double* Gr = g.G + ro * Bn;
#pragma unroll 4
      for (int j = kk; j < Bn; j += ks) acc = fma(-Gr[j], g.xb[j * B + sh], acc);
    }
    acc = lane_group_sum(acc, ks);
    if (live && kk == 0) a.x[(int64_t)g.sep[ro] * B + sh] = acc;
  }
}

// the same for a small front done by one warp (all rows; no block synchronisation)
__device__ void fwd_compute_warp(const SolveArgs& a, const Task& tk, const double* sm, int lane) {
  const int B = a.B, S = tk.s;
  const FwdStage f = fwd_layout(tk, const_cast<double*>(sm), B);
  const double* csep = f.vals;
  const double* cb = f.vals + (size_t)S * B;
  const int n = f.rows * B;
  for (int o = lane; o < n; o += 32) {
    const int r = div_shots(a, o), sh = o - r * B;
    double acc = 0.0;
    for (int k = 0; k < S; ++k) acc = fma(f.C[r * S + k], csep[k * B + sh], acc);
    a.ybnd[tk.bnd_off * B + o] = cb[o] - acc;
  }
}

__device__ void bwd_compute_warp(const SolveArgs& a, const Task& tk, const double* sm, int lane) {
  const int B = a.B, S = tk.s, Bn = tk.b;
  const BwdStage g = bwd_layout(tk, const_cast<double*>(sm), B);
  for (int o = lane; o < g.rows * B; o += 32) {
    const int r = div_shots(a, o), sh = o - r * B;
    double acc = 0.0;
    for (int k = 0; k < S; ++k) acc = fma(g.X[r * S + k], g.ys[k * B + sh], acc);
    for (int j = 0; j < Bn; ++j) acc = fma(-g.G[r * Bn + j], g.xb[j * B + sh], acc);
    a.x[(int64_t)g.sep[r] * B + sh] = acc;
  }
}

// A whole task with nothing to wait for (the barrier and per-level schedules).  Block
// tasks end with __syncthreads (the staging area is reused by the block's next task),
// warp tasks with __syncwarp.
__device__ void solve_forward_task(const SolveArgs& a, const Task tk, double* sm) {
  fwd_stage_all<8>(a, tk, sm, tk.r0 == 0, threadIdx.x, blockDim.x);
  __syncthreads();
  fwd_compute_block(a, tk, sm);
  __syncthreads();
}

__device__ void solve_backward_task(const SolveArgs& a, const Task tk, double* sm) {
  bwd_stage_all<8>(a, tk, sm, threadIdx.x, blockDim.x);
  __syncthreads();
  bwd_compute_block(a, tk, sm);
  __syncthreads();
}

__device__ void solve_forward_warp(const SolveArgs& a, const Task tk, double* sm, int lane) {
  fwd_stage_all<8>(a, tk, sm, true, lane, 32);
  __syncwarp();
  fwd_compute_warp(a, tk, sm, lane);
  __syncwarp();
}

__device__ void solve_backward_warp(const SolveArgs& a, const Task tk, double* sm, int lane) {
  bwd_stage_all<8>(a, tk, sm, lane, 32);
  __syncwarp();
  bwd_compute_warp(a, tk, sm, lane);
  __syncwarp();
}

// The work of one tree level in one direction, as block items: tasks [start, wstart)
// are block tasks, [wstart, end) warp tasks taken `group` at a time.  Block items
// come first, so once a block reaches the warp items its warps only touch their
// own shared-memory slices.
__device__ void run_level(const SolveArgs& a, const Task* tasks, const int32_t* meta, int levels, int l, bool fwd,
                          double* sm, int item0, int stride) {
  const int start = meta[l], end = meta[l + 1], wstart = meta[levels + 1 + l], group = meta[2 * levels + 1 + l];
  const int nblock = wstart - start;
  const int nitems = nblock + (end - wstart + group - 1) / group;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int it = item0; it < nitems; it += stride) {
    if (it < nblock) {
      if (fwd) solve_forward_task(a, tasks[start + it], sm);
      else solve_backward_task(a, tasks[start + it], sm);
    } else {
      const int w = wstart + (it - nblock) * group + warp;
      if (warp < group && w < end) {
        double* wsm = sm + (size_t)warp * a.warp_doubles;
        if (fwd) solve_forward_warp(a, tasks[w], wsm, lane);
        else solve_backward_warp(a, tasks[w], wsm, lane);
      }
    }
  }
}

struct LevelKernelArgs {
  SolveArgs s;
  const Task* tasks;
  const int32_t* meta;
  int levels, level;
};

__global__ void __launch_bounds__(256) solve_forward_kernel(LevelKernelArgs a) {
  extern __shared__ double sm_fwd[];
  run_level(a.s, a.tasks, a.meta, a.levels, a.level, true, sm_fwd, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) solve_backward_kernel(LevelKernelArgs a) {
  extern __shared__ double sm_bwd[];
  run_level(a.s, a.tasks, a.meta, a.levels, a.level, false, sm_bwd, blockIdx.x, gridDim.x);
}


struct PersistentSolveArgs {
  SolveArgs s;
  const Task* fwd;
  const Task* bwd;
  const int32_t* fwd_meta;    // start[L+1] | wstart[L] | group[L]
  const int32_t* bwd_meta;
  int levels;
  unsigned* bar;              // [2]: arrival count, generation
  int* status;
  long long budget;
  unsigned long long* trace;   // nullable: per-level wall time accumulators (block 0)
};

// the whole boundary solve of one time step: forward pass leaves -> root, then
// backward pass root -> leaves, one grid barrier between tree levels
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(256, 4) solve_persistent_kernel(PersistentSolveArgs a) {
  extern __shared__ double sm_p[];
  // trace (profiling only): [0, 2L) wall time per phase seen by block 0, [2L, 4L) the
  // longest time any block spent in its tasks of the phase, [4L, 6L) the sum over
  // blocks of that time
  const int L2 = 2 * a.levels;
  const bool tr = a.trace && threadIdx.x == 0;
  unsigned long long t_prev = tr ? global_ns() : 0ULL, t_start = t_prev;
  int slot = 0;
  auto busy = [&]() {
    if (tr) {
      const unsigned long long d = global_ns() - t_start;
      atomicMax(a.trace + L2 + slot, d);
      atomicAdd(a.trace + 2 * L2 + slot, d);
    }
  };
  auto mark = [&]() {
    if (tr) {
      const unsigned long long t = global_ns();
      if (blockIdx.x == 0) a.trace[slot] += t - t_prev;
      t_prev = t;
      t_start = t;
    }
    ++slot;
  };
  for (int l = 0; l < a.levels; ++l) {
    run_level(a.s, a.fwd, a.fwd_meta, a.levels, l, true, sm_p, blockIdx.x, gridDim.x);
    busy();
    if (!grid_barrier(a.bar, a.bar + 1, a.status, a.budget)) return;
    mark();
  }
  for (int l = a.levels - 1; l >= 0; --l) {
    run_level(a.s, a.bwd, a.bwd_meta, a.levels, l, false, sm_p, blockIdx.x, gridDim.x);
    busy();
    if (l > 0 && !grid_barrier(a.bar, a.bar + 1, a.status, a.budget)) return;
    mark();              // the last one: block 0's own finish
  }
}

// ---------------------------------------------------------------------------
// the same solve as a dataflow: no grid barriers.  Blocks claim work items in a
// topological order (forward items leaves -> root, then backward items root ->
// leaves) from one counter; an item waits only for the tasks it reads from: a
// forward task for every forward task of its children, a backward task for the
// forward tasks of its own node and the backward tasks of its nearest ancestor that
// has any.  Counters are cumulative over the launches of one time loop: after g
// solves a node has g * n tasks done.  Every dependency of an item lies in an item
// claimed earlier and all blocks are co-resident, so the earliest unfinished claimed
// item can always proceed; every wait is still bounded and reports SBFWI_ETIMEOUT.
// ---------------------------------------------------------------------------
struct FlowArgs {
  SolveArgs s;
  const Task* fwd;
  const Task* bwd;
  const int4* items;          // {first task, count, block (1) or warp group (0), direction (0 fwd, 1 bwd)}
  int n_items;
  const int32_t* node_info;   // [5][nodes]: forward tasks, backward tasks, child0, child1, backward dependency
  int nodes;
  unsigned* done_f;           // [nodes] forward tasks completed (cumulative)
  unsigned* done_b;           // [nodes] backward tasks completed (cumulative)
  unsigned long long* claim;  // item counter (cumulative)
  unsigned long long base;    // counter value at the start of this launch
  unsigned gen;               // this launch's number in the time loop, from 1
  int* status;
  long long budget;
  int levels;
  unsigned long long* trace;  // nullable: this solve's row of the per-phase trace (profiling)
};

// profiling: one item of phase `ph` finished (timer values of its claim and of its inputs
// being ready)
__device__ __forceinline__ void flow_record(const FlowArgs& a, int ph, unsigned long long t_claim,
                                            unsigned long long t_ready) {
  const unsigned long long t = global_ns();
  unsigned long long* f = a.trace + 1 + 4 * ph;
  atomicMax(f, t);
  atomicAdd(f + 1, t - t_ready);
  atomicAdd(f + 2, t_ready - t_claim);
  atomicAdd(f + 3, 1ULL);
}

// completion counter update: a release, so every write of the task (ordered before it by
// the block or warp barrier) is visible to a thread whose acquire load sees the new count
__device__ __forceinline__ void add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// one thread: wait until counter >= target (an acquire: the producers' writes before
// their counter update are visible after it); false if the budget ran out or another
// wait gave up
__device__ bool wait_count(const unsigned* counter, unsigned target, int* status, long long budget) {
  if (ld_acquire(counter) >= target) return true;
  const long long t0 = clock64();
  while (ld_acquire(counter) < target) {
    if (clock64() - t0 > budget || *(volatile int*)status != 0) {
      atomicCAS(status, 0, SBFWI_ETIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// A forward task reads its children's boundaries: every forward task of both children.
__device__ bool wait_children(const FlowArgs& a, int node) {
  const int T = a.nodes;
  const int32_t* nf = a.node_info;
  const int ch[2] = {a.node_info[2 * T + node], a.node_info[3 * T + node]};
  bool ok = true;
  for (int k = 0; k < 2 && ok; ++k)
    if (ch[k] >= 0) ok = wait_count(a.done_f + ch[k], a.gen * (unsigned)nf[ch[k]], a.status, a.budget);
  return ok;
}

// A backward task reads y_sep of its own node (that node's forward tasks) ...
__device__ bool wait_own(const FlowArgs& a, int node) {
  return wait_count(a.done_f + node, a.gen * (unsigned)a.node_info[node], a.status, a.budget);
}

// ... and x at its boundary: the backward tasks of its nearest ancestor that has any.
__device__ bool wait_ancestor(const FlowArgs& a, int node) {
  const int T = a.nodes;
  const int d = a.node_info[4 * T + node];
  return d < 0 || wait_count(a.done_b + d, a.gen * (unsigned)a.node_info[T + d], a.status, a.budget);
}

// kTrace: the profiling variant that stamps the timer (a.trace set); the other ignores a.trace
template <bool kTrace>
__global__ void __launch_bounds__(256, 4) solve_flow_kernel(FlowArgs a) {
  extern __shared__ double sm_f[];
  __shared__ long long s_item;
  __shared__ int s_ok[2];
  __shared__ unsigned long long s_tclaim;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool tr = kTrace;
  if (tr && threadIdx.x == 0) atomicMin(a.trace, global_ns());
  for (;;) {
    // a wait that gave up anywhere stops every block at its next claim
    if (threadIdx.x == 0) {
      s_item = *(volatile int*)a.status != 0 ? (long long)a.n_items
                                            : (long long)(atomicAdd(a.claim, 1ULL) - a.base);
      if (tr) s_tclaim = global_ns();
    }
    __syncthreads();
    const long long it = s_item;
    __syncthreads();
    if (it >= a.n_items) return;
    const int4 im = a.items[it];
    const Task* tasks = im.w ? a.bwd : a.fwd;
    unsigned long long t_ready = tr ? s_tclaim : 0ULL;     // profiling: when the inputs were ready
    if (im.z == 1) {                                       // block task
      const Task tk = tasks[im.x];
      // what does not depend on other tasks first: it hides its latency behind the waits
      if (im.w) {
        bwd_stage_const<8>(a.s, tk, sm_f, threadIdx.x, blockDim.x);
        if (threadIdx.x == 0) s_ok[0] = wait_own(a, tk.node) ? 1 : 0;
        __syncthreads();
        if (!s_ok[0]) return;
        bwd_stage_own<8>(a.s, tk, sm_f, threadIdx.x, blockDim.x);
        if (threadIdx.x == 0) s_ok[1] = wait_ancestor(a, tk.node) ? 1 : 0;
        __syncthreads();
        if (!s_ok[1]) return;
        if (tr && threadIdx.x == 0) t_ready = global_ns();
        bwd_stage_data<8>(a.s, tk, sm_f, threadIdx.x, blockDim.x);
        __syncthreads();
        bwd_compute_block(a.s, tk, sm_f);
      } else {
        fwd_stage_const<8>(a.s, tk, sm_f, threadIdx.x, blockDim.x);
        if (threadIdx.x == 0) s_ok[0] = wait_children(a, tk.node) ? 1 : 0;
        __syncthreads();
        if (!s_ok[0]) return;
        if (tr && threadIdx.x == 0) t_ready = global_ns();
        fwd_stage_data<8>(a.s, tk, sm_f, tk.r0 == 0, threadIdx.x, blockDim.x);
        __syncthreads();
        fwd_compute_block(a.s, tk, sm_f);
      }
      __syncthreads();     // every output stored; the staging area is free for the next item
      if (threadIdx.x == 0) {
        add_release((im.w ? a.done_b : a.done_f) + tk.node, 1u);
        if (tr) flow_record(a, im.w * a.levels + (tk.pad & 0xff), s_tclaim, t_ready);
      }
    } else if (warp < im.y) {                              // warp task
      const Task tk = tasks[im.x + warp];
      double* wsm = sm_f + (size_t)warp * a.s.warp_doubles;
      int ok = 1;
      if (im.w) {
        bwd_stage_const<8>(a.s, tk, wsm, lane, 32);
        if (lane == 0) ok = wait_own(a, tk.node) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
          bwd_stage_own<8>(a.s, tk, wsm, lane, 32);
          if (lane == 0) ok = wait_ancestor(a, tk.node) ? 1 : 0;
          ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (ok) {
          if (tr && lane == 0) t_ready = global_ns();
          __syncwarp();
          bwd_stage_data<8>(a.s, tk, wsm, lane, 32);
          __syncwarp();
          bwd_compute_warp(a.s, tk, wsm, lane);
        }
      } else {
        fwd_stage_const<8>(a.s, tk, wsm, lane, 32);
        if (lane == 0) ok = wait_children(a, tk.node) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (ok) {
          if (tr && lane == 0) t_ready = global_ns();
          __syncwarp();
          fwd_stage_data<8>(a.s, tk, wsm, true, lane, 32);
          __syncwarp();
          fwd_compute_warp(a.s, tk, wsm, lane);
        }
      }
      __syncwarp();
      if (ok && lane == 0) {                               // else: the status stops the block at its next claim
        add_release((im.w ? a.done_b : a.done_f) + tk.node, 1u);
        if (tr) flow_record(a, im.w * a.levels + (tk.pad & 0xff), s_tclaim, t_ready);
      }
    }
  }
}

// Self-test of the bounded grid barrier: blocks with index >= gridDim.x - absent
// return at once and never arrive, so with absent > 0 every other block gives up
// after `budget` cycles and the status reads SBFWI_ETIMEOUT.
__global__ void barrier_selftest_kernel(unsigned* bar, int* status, long long budget, int absent, int rounds) {
  if ((int)blockIdx.x >= (int)gridDim.x - absent) return;
  for (int r = 0; r < rounds; ++r)
    if (!grid_barrier(bar, bar + 1, status, budget)) return;
}

// ---------------------------------------------------------------------------
// boundary nodes: Newmark update, receivers, store / gradient
// ---------------------------------------------------------------------------
struct BoundaryArgs {
  int64_t N;
  int B, R;
  int64_t K, k;
  double a0, a1, a2, c1, c2, dt;
  const double* x;
  double* ub; double* udb; double* uddb;
  const int64_t* rec;
  double* traces;         // [B][R][K]
  double* store_b;        // forward: velocities of this step at the boundary nodes [N][B]
  double* store_ub;       // forward, full kernel / exact adjoint: displacements of this step at the boundary nodes [N][B]
  double* store_ab;       // forward, exact adjoint: accelerations of this step at the boundary nodes [N][B]
  const double* fwd_b;    // adjoint: paired forward velocities [N][B]
  double* grad_b;         // adjoint accumulators [N][B]
};

__global__ void boundary_update_kernel(BoundaryArgs a) {
  const int64_t tot = a.N * a.B;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const double un = a.x[t];
    const double uo = a.ub[t], udo = a.udb[t], uddo = a.uddb[t];
    const double vo = fma(a.a0, uo, fma(a.a1, udo, a.a2 * uddo));
    const double uddn = fma(a.a0, un, -vo);
    const double udn = fma(a.c2, uddn, fma(a.c1, uddo, udo));
    a.ub[t] = un; a.udb[t] = udn; a.uddb[t] = uddn;
    if (a.store_b) a.store_b[t] = udn;
    if (a.store_ub) a.store_ub[t] = un;
    if (a.store_ab) a.store_ab[t] = uddn;
    if (a.grad_b) a.grad_b[t] = fma(a.fwd_b[t], udn, a.grad_b[t]);          // dt applied at the end
  }
  if (a.traces) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)a.R * a.B; t += (int64_t)gridDim.x * blockDim.x) {
      const int s = (int)(t / a.R), r = (int)(t - (int64_t)s * a.R);
      a.traces[((int64_t)s * a.R + r) * a.K + a.k] = a.x[a.rec[r] * a.B + s];
    }
  }
}

// external sources of one step: forward wavelets at the source nodes, or the
// time-reversed residuals at the receivers
__global__ void sources_kernel(double* ext, int B, int nsrc, const int64_t* node, const double* values,
                               int64_t stride_src, int64_t col, int per_shot) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * nsrc) return;
  const int s = t / nsrc, j = t - s * nsrc;
  // per_shot: one source per shot (node[s]); otherwise nsrc receivers shared by all shots
  const int64_t g = per_shot ? node[s] : node[j];
  ext[g * B + s] = values[(per_shot ? (int64_t)s : ((int64_t)s * nsrc + j)) * stride_src + col];
}

// ---------------------------------------------------------------------------
// gradient: shots summed, then optionally the transpose of the bilinear map
// ---------------------------------------------------------------------------
// g(node) = dt * sum over shots of the accumulated sum_m udot_fwd * lambdadot
__global__ void sum_shots_kernel(const double* acc, int64_t np, int B, double dt, double* out, int accumulate) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np; q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += acc[q * B + b];
    s *= dt;
    out[q] = accumulate ? out[q] + s : s;
  }
}

// Comparison method (low-frequency expansion): the effective source of every element for
// the next step, f_hat_e = M_e (a0 u + a1 u' + a2 u'') at its boundary nodes, so that the
// global system (sum of K_e + a0 M_e) u = f + sum f_hat_e is Newmark on M u'' + K u = f.
__global__ void lfe_source_kernel(const double* M, const int32_t* dofs, const double* ub, const double* udb,
                                  const double* uddb, int64_t E, int nb, int B, double a0, double a1, double a2,
                                  double* fhat) {
  const int64_t tot = E * nb * B;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / ((int64_t)nb * B);
    const int r = (int)((t / B) % nb), s = (int)(t % B);
    const double* Mr = M + (e * nb + r) * (int64_t)nb;
    double acc = 0.0;
    for (int c = 0; c < nb; ++c) {
      const int64_t g = (int64_t)dofs[e * nb + c] * B + s;
      acc = fma(Mr[c], fma(a0, ub[g], fma(a1, udb[g], a2 * uddb[g])), acc);
    }
    fhat[t] = acc;
  }
}

// out[q] (+)= lib[map[q]]: nodal values from the padded layout to the caller's
// Gradient term of the full Frechet kernel at one adjoint step, for every nodal point q and
// shot s: grad[q][s] += c^2 (G u_fwd)(q, s) . (G lambda)(q, s), G the nodal gradient operator
// (CSR rows 2q, 2q+1); lambda's interior part from lam_int, its boundary part from lam_b.
// dt is applied at the end with the velocity term.
__global__ void gradient_term_kernel(const int64_t* ptr, const int32_t* col, const double* val, int64_t np,
                                     int64_t n_int, int B, const double* u_fwd, const double* lam_int,
                                     const double* lam_b, double c2, double* grad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < np * B; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / B;
    const int s = (int)(t - q * B);
    double gu[2], gl[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      double au = 0.0, al = 0.0;
      for (int64_t k = ptr[2 * q + d]; k < ptr[2 * q + d + 1]; ++k) {
        const int64_t c = col[k];
        const double v = val[k];
        au = fma(v, u_fwd[c * B + s], au);
        al = fma(v, c < n_int ? lam_int[c * B + s] : lam_b[(c - n_int) * B + s], al);
      }
      gu[d] = au;
      gl[d] = al;
    }
    grad[t] = fma(c2, fma(gu[0], gl[0], gu[1] * gl[1]), grad[t]);
  }
}

__global__ void gather_nodal_kernel(const double* lib, const int64_t* map, int64_t n, double* out, int accumulate) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = accumulate ? out[q] + lib[map[q]] : lib[map[q]];
}

__global__ void grid_transpose_kernel(const double* g_nodal, const double* pts, const int32_t* cell_of_point,
                                      const int8_t* clamp, const int64_t* cell_ptr, const int64_t* cell_list,
                                      int64_t gx, int64_t gy, double lx, double ly, double* out, int accumulate) {
  const int64_t ncell = gx * gy;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t l = cell_ptr[c]; l < cell_ptr[c + 1]; ++l) {
      const int64_t q = cell_list[l] >> 2;
      const int k = (int)(cell_list[l] & 3);
      const int32_t base = cell_of_point[q];
      const int64_t ix = base % gx, iy = base / gx;
      const int8_t cl = clamp[q];
      double tx = (cl & 1) ? 0.0 : (cl & 2) ? 1.0 : pts[2 * q] * gx / lx - 0.5 - (double)ix;
      double ty = (cl & 4) ? 0.0 : (cl & 8) ? 1.0 : pts[2 * q + 1] * gy / ly - 0.5 - (double)iy;
      const double wx = (k & 1) ? tx : 1.0 - tx;
      const double wy = (k >> 1) ? ty : 1.0 - ty;
      acc = fma(wx * wy, g_nodal[q], acc);
    }
    out[c] = accumulate ? out[c] + acc : acc;
  }
}

// the same for a 3-D grid (trilinear weights, cell_list entries point * 8 + corner)
__global__ void grid_transpose3d_kernel(const double* g_nodal, const double* pts, const int32_t* cell_of_point,
                                        const int8_t* clamp, const int64_t* cell_ptr, const int64_t* cell_list,
                                        int64_t gx, int64_t gy, int64_t gz, double lx, double ly, double lz,
                                        double* out, int accumulate) {
  const int64_t ncell = gx * gy * gz;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t l = cell_ptr[c]; l < cell_ptr[c + 1]; ++l) {
      const int64_t q = cell_list[l] >> 3;
      const int k = (int)(cell_list[l] & 7);
      const int64_t base = cell_of_point[q];
      const int64_t b3[3] = {base % gx, (base / gx) % gy, base / (gx * gy)};
      const int64_t g3[3] = {gx, gy, gz};
      const double l3[3] = {lx, ly, lz};
      const int8_t cl = clamp[q];
      double w = 1.0;
      for (int d = 0; d < 3; ++d) {
        const double t = (cl & (1 << (2 * d))) ? 0.0 : (cl & (2 << (2 * d))) ? 1.0
                                                     : pts[3 * q + d] * g3[d] / l3[d] - 0.5 - (double)b3[d];
        w *= ((k >> d) & 1) ? t : 1.0 - t;
      }
      acc = fma(w, g_nodal[q], acc);
    }
    out[c] = accumulate ? out[c] + acc : acc;
  }
}

// ---------------------------------------------------------------------------
// misfit (deterministic two-pass reduction)
// ---------------------------------------------------------------------------
__global__ void misfit_partial_kernel(const double* tr, const double* ob, int64_t n, double* res, double* partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double d = ob[t] - tr[t];
    if (res) res[t] = d;
    acc = fma(d, d, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void misfit_final_kernel(const double* partial, int nparts, double half_dt, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) acc += partial[t];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = half_dt * red[0];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int pow2_ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}
static int pow2_floor(int v) {
  int p = 1;
  while (2 * p <= v) p <<= 1;
  return p;
}

// Small fronts (s <= kWarpS, b <= kWarpB) are warp tasks: one warp does every row.
static constexpr int kWarpS = 8, kWarpB = 32;
static bool warp_front(const TreeNodeDev& r) { return r.s <= kWarpS && r.b <= kWarpB; }
// staging area of one warp task: vectors (s + b) B, the factors s (s + b) and the node
// ids or source rows (at most 2 (s + b) int32)
size_t solve_warp_doubles(int B) {
  return (size_t)(kWarpS + kWarpB) * (B + 1) + (size_t)kWarpS * (kWarpS + kWarpB);
}
// staging area of a block task (the layouts of fwd_layout / bwd_layout)
static size_t block_task_doubles(const Task& t, int B, bool fwd) {
  const size_t rows = (size_t)(t.r1 - t.r0);
  return fwd ? (t.s + rows) * B + rows * t.s + (t.s + rows)
             : (size_t)(t.s + t.b) * B + rows * (t.s + t.b) + (t.b + rows + 1) / 2;
}

// B shots, `grid` blocks.  Block tasks of a level take a power-of-two number of rows
// chosen so that the level's rows about fill the grid (the top of the tree has few,
// long rows: one row per block, its dot products split over up to 32 lanes); the
// lanes per output fill the block's 256 threads.  Leaves that eliminate nothing get
// no task (their parents read f_hat directly).  Warp tasks are grouped so that a
// level's items about fill the grid.
int build_level_tasks(const Model& md, LevelTasks& lt, int B, int grid) {
  // rows x shots <= 256 outputs per block task (one per thread); 512 on levels whose separators
  // are at most 32 nodes (their factor rows are short, so the staging stays small)
  const int rows_max = std::max(1, 256 / B), rows_max_short = std::max(1, 512 / B);
  const Tree& t = md.mesh->tree;
  const int L = t.levels;
  std::vector<Task> fwd, bwd;
  lt.fwd_start.assign(L + 1, 0); lt.bwd_start.assign(L + 1, 0);
  lt.fwd_wstart.assign(L, 0); lt.bwd_wstart.assign(L, 0);
  lt.fwd_group.assign(L, 1); lt.bwd_group.assign(L, 1);
  auto task = [&](int32_t nd, int32_t r0, int32_t r1, int ks) {
    const TreeNodeDev& r = t.nodes[nd];
    Task tk;
    tk.node = nd; tk.r0 = r0; tk.r1 = r1; tk.ksplit = ks;
    tk.s = r.s; tk.b = r.b; tk.leaf = r.elem >= 0 ? 1 : 0; tk.pad = t.level_of[nd];   // height: the trace's phase
    tk.sep_off = r.sep_off; tk.bnd_off = r.bnd_off; tk.map_off = r.map_off; tk.X_off = r.X_off;
    return tk;
  };
  auto group_for = [&](int n) { return std::max(1, std::min(8, (n + grid - 1) / std::max(grid, 1))); };
  // rows per block task and lanes per output for a dot product of length len
  auto rows_for = [&](int64_t level_rows, int cap) {
    const int64_t per = (level_rows + grid - 1) / std::max(grid, 1);
    return std::min(cap, pow2_ceil((int)std::max<int64_t>(1, per)));
  };
  auto lanes_for = [&](int rows, int len) {
    return std::max(1, std::min({32, pow2_floor(std::max(1, 256 / (B * rows))), pow2_ceil(std::max(1, len))}));
  };
  for (int l = 0; l < L; ++l) {
    lt.fwd_start[l] = (int32_t)fwd.size();
    lt.bwd_start[l] = (int32_t)bwd.size();
    int64_t rows_f = 0, rows_b = 0;
    int s_max = 0;
    for (int32_t nd : t.nodes_at_level[l]) {
      const TreeNodeDev& r = t.nodes[nd];
      if (!warp_front(r)) { rows_f += r.b; rows_b += r.s; s_max = std::max(s_max, (int)r.s); }
    }
    const int rf = rows_for(rows_f, s_max <= 32 ? rows_max_short : rows_max), rb = rows_for(rows_b, rows_max);
    for (int32_t nd : t.nodes_at_level[l]) {
      const TreeNodeDev& r = t.nodes[nd];
      if (warp_front(r)) continue;
      const int kf = lanes_for(rf, r.s), kb = lanes_for(rb, r.s + r.b);
      if (r.b == 0) fwd.push_back(task(nd, 0, 0, 1));
      for (int32_t r0 = 0; r0 < r.b; r0 += rf) fwd.push_back(task(nd, r0, std::min(r.b, r0 + rf), kf));
      for (int32_t r0 = 0; r0 < r.s; r0 += rb) bwd.push_back(task(nd, r0, std::min(r.s, r0 + rb), kb));
    }
    lt.fwd_wstart[l] = (int32_t)fwd.size();
    lt.bwd_wstart[l] = (int32_t)bwd.size();
    for (int32_t nd : t.nodes_at_level[l]) {
      const TreeNodeDev& r = t.nodes[nd];
      if (!warp_front(r)) continue;
      // a leaf that eliminates nothing passes f_hat through (its parent reads f_hat)
      if (!(r.elem >= 0 && r.s == 0)) fwd.push_back(task(nd, 0, r.b, 1));
      if (r.s > 0) bwd.push_back(task(nd, 0, r.s, 1));
    }
    lt.fwd_group[l] = group_for((int)fwd.size() - lt.fwd_wstart[l]);
    lt.bwd_group[l] = group_for((int)bwd.size() - lt.bwd_wstart[l]);
  }
  lt.fwd_start[L] = (int32_t)fwd.size();
  lt.bwd_start[L] = (int32_t)bwd.size();
  lt.block_doubles = 1;
  for (int l = 0; l < L; ++l) {
    for (int k = lt.fwd_start[l]; k < lt.fwd_wstart[l]; ++k)
      lt.block_doubles = std::max(lt.block_doubles, block_task_doubles(fwd[k], B, true));
    for (int k = lt.bwd_start[l]; k < lt.bwd_wstart[l]; ++k)
      lt.block_doubles = std::max(lt.block_doubles, block_task_doubles(bwd[k], B, false));
  }
  lt.max_level_items = 1;
  for (int l = 0; l < L; ++l) lt.max_level_items = std::max({lt.max_level_items, lt.items(true, l), lt.items(false, l)});
  // dataflow items: forward levels leaves -> root, then backward levels root -> leaves
  {
    std::vector<int4> items;
    auto add_level = [&](const std::vector<int32_t>& st, const std::vector<int32_t>& ws,
                         const std::vector<int32_t>& gr, int l, int dir) {
      for (int k = st[l]; k < ws[l]; ++k) items.push_back(make_int4(k, 1, 1, dir));
      for (int k = ws[l]; k < st[l + 1]; k += gr[l]) items.push_back(make_int4(k, std::min(gr[l], st[l + 1] - k), 0, dir));
    };
    // the lower levels whose block tasks fit the warp tasks' staging area run at full
    // occupancy in their own launches; a few large fronts at the top (3-D separators are
    // planes) then no longer hold the whole solve at one block per SM
    lt.small_doubles = 8 * solve_warp_doubles(B);
    int low = -1;                                  // levels 0..low fit
    for (int l = 0; l < L; ++l) {
      size_t dl = 0;
      for (int k = lt.fwd_start[l]; k < lt.fwd_wstart[l]; ++k) dl = std::max(dl, block_task_doubles(fwd[k], B, true));
      for (int k = lt.bwd_start[l]; k < lt.bwd_wstart[l]; ++k) dl = std::max(dl, block_task_doubles(bwd[k], B, false));
      if (dl > lt.small_doubles) break;
      low = l;
    }
    for (int l = 0; l < L; ++l) {
      if (l == low + 1) lt.flow_seg[1] = (int)items.size();
      add_level(lt.fwd_start, lt.fwd_wstart, lt.fwd_group, l, 0);
    }
    if (low + 1 >= L) lt.flow_seg[1] = (int)items.size();
    for (int l = L - 1; l >= 0; --l) {
      if (l == low) lt.flow_seg[2] = (int)items.size();
      add_level(lt.bwd_start, lt.bwd_wstart, lt.bwd_group, l, 1);
    }
    lt.flow_seg[0] = 0;
    lt.flow_seg[3] = (int)items.size();
    if (low < 0) lt.flow_seg[2] = lt.flow_seg[3];                      // no level fits: one launch
    if (low + 1 >= L) lt.flow_seg[1] = lt.flow_seg[2] = lt.flow_seg[3];   // every level fits: one launch
    const int T = (int)t.nodes.size();
    std::vector<int32_t> info(5 * (size_t)T, 0), parent(T, -1);
    for (const Task& tk : fwd) info[tk.node] += 1;
    for (const Task& tk : bwd) info[T + tk.node] += 1;
    for (int nd = 0; nd < T; ++nd) {
      info[2 * T + nd] = t.nodes[nd].child0;
      info[3 * T + nd] = t.nodes[nd].child1;
      if (t.nodes[nd].child0 >= 0) parent[t.nodes[nd].child0] = nd;
      if (t.nodes[nd].child1 >= 0) parent[t.nodes[nd].child1] = nd;
    }
    for (int nd = 0; nd < T; ++nd) {
      int a = parent[nd];
      while (a >= 0 && info[T + a] == 0) a = parent[a];
      info[4 * T + nd] = a;
    }
    SBFWI_CUDA(lt.flow_items.alloc(sizeof(int4) * std::max<size_t>(items.size(), 1)));
    if (!items.empty())
      SBFWI_CUDA(cudaMemcpy(lt.flow_items.p, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    SBFWI_CUDA(lt.node_info.alloc(sizeof(int32_t) * info.size()));
    SBFWI_CUDA(cudaMemcpy(lt.node_info.p, info.data(), sizeof(int32_t) * info.size(), cudaMemcpyHostToDevice));
    lt.n_items = (int)items.size();
    lt.nodes = T;
  }
  auto upload_meta = [&](DevBuf& dst, const std::vector<int32_t>& st, const std::vector<int32_t>& ws,
                         const std::vector<int32_t>& gr) -> int {
    std::vector<int32_t> meta(st);
    meta.insert(meta.end(), ws.begin(), ws.end());
    meta.insert(meta.end(), gr.begin(), gr.end());
    SBFWI_CUDA(dst.alloc(sizeof(int32_t) * meta.size()));
    SBFWI_CUDA(cudaMemcpy(dst.p, meta.data(), sizeof(int32_t) * meta.size(), cudaMemcpyHostToDevice));
    return SBFWI_OK;
  };
  int rc = upload_meta(lt.fwd_meta, lt.fwd_start, lt.fwd_wstart, lt.fwd_group);
  if (rc) return rc;
  rc = upload_meta(lt.bwd_meta, lt.bwd_start, lt.bwd_wstart, lt.bwd_group);
  if (rc) return rc;
  SBFWI_CUDA(lt.fwd.alloc(sizeof(Task) * std::max<size_t>(fwd.size(), 1)));
  SBFWI_CUDA(lt.bwd.alloc(sizeof(Task) * std::max<size_t>(bwd.size(), 1)));
  if (!fwd.empty()) SBFWI_CUDA(cudaMemcpy(lt.fwd.p, fwd.data(), sizeof(Task) * fwd.size(), cudaMemcpyHostToDevice));
  if (!bwd.empty()) SBFWI_CUDA(cudaMemcpy(lt.bwd.p, bwd.data(), sizeof(Task) * bwd.size(), cudaMemcpyHostToDevice));
  lt.shots = B;
  lt.grid = grid;
  return SBFWI_OK;
}

namespace {

struct RunBuffers {
  DevBuf u, ud, udd, v, ub, udb, uddb, q, fhat, ext, ysep, ybnd, x;
  DevBuf lam;                       // full kernel, adjoint: interior displacements of the current step
  DevBuf grad_int;                  // grad accumulators [n_nodal][B] (adjoint)
  // exact adjoint: mu of rows -1..n, v_bar_n per element, ghosts of the forward solution,
  // Gauss-point products, boundary station of the gradient per element
  DevBuf mu, vbn, ghost, gacc, gbnd;
};

// Forward: the forward solve; Adjoint: the paper's time-reversed adjoint with the velocity
// kernel; Exact: the exact discrete adjoint (transposed condensation, transposed global
// solve, Gauss-point products of the derivative of every block)
enum class Mode { Forward, Adjoint, Exact };

// The time loop of B shots over K Newmark steps, resumable over windows of steps.
// Forward: values = wavelets [B][K] at nodes[0..B-1], receivers nodes[B..B+R-1];
// writes traces and (if `store`) the nodal velocities of every step it runs.
// Adjoint: values = residuals [B][R][K] at nodes[0..R-1], injected last sample
// first; accumulates the correlation with the forward velocities in `fwd` into
// grad_int [n_nodal][B].
//
// run(k0, k1) takes steps k0..k1-1 and ends with the back-substitution of step
// k1-1, so between two windows the state is the complete Newmark state after
// step k0-1: {u or v, u', u''} of the interior and {u, u', u''} of the boundary
// nodes.  A window that starts at k0 > 0 first runs the forward sweep of step k0
// from that state.  Splitting the fused element launch at a window edge gives the
// same values bit for bit (the two halves compute exactly what the fused launch
// does), so a run cut into windows, or resumed from a saved state, reproduces the
// uncut run.
struct Stepper {
  Model& md;
  const Mode mode;
  const int B, R;
  const int64_t K;
  RunBuffers& rb;
  const cudaStream_t st;
  // forward: velocities of step k go to store + (k - store_k0) * n_nodal * B
  double* store = nullptr;
  double* store_u = nullptr;        // full kernel: displacements of step k at store_u + (k - store_k0) * n_nodal * B
  double* store_a = nullptr;        // exact adjoint: accelerations of step k, paired like store_u
  int64_t store_k0 = 0;
  // adjoint: forward velocities of step j are read at fwd + (j - fwd_k0) * n_nodal * B
  const double* fwd = nullptr;
  const double* fwd_u = nullptr;    // full kernel and exact adjoint: forward displacements, paired like fwd
  const double* fwd_a = nullptr;    // exact adjoint: forward accelerations of step j at fwd_a + (j - fwd_k0) * n_nodal * B
  int64_t fwd_k0 = 0;
  // source values and nodes (forward: wavelets [B][K], nodes = B sources then R
  // receivers; adjoint: residuals [B][R][K], nodes = R receivers) and the device
  // traces [B][R][K] (forward with R > 0)
  const double* values = nullptr;
  const int64_t* nodes = nullptr;
  double* traces = nullptr;

  // the solve's task lists: the model's (shared by the steppers of one call), or the
  // caller's own when this stepper outlives a call (a session: a later call with another
  // shot count rebuilds the model's)
  LevelTasks* tasks_own = nullptr;
  // resume: the window that run(0, k1) starts continues a nonzero state (the forward sweep
  // of its first step is computed from it)
  bool resume = false;

  Stepper(Model& m, Mode mo, int b, int64_t k, int r, RunBuffers& buffers, cudaStream_t s)
      : md(m), mode(mo), B(b), R(r), K(k), rb(buffers), st(s) {}

  int init();
  int zero_state();
  int run(int64_t k0, int64_t k1);
  // exact adjoint: forward steps k1-1 down to k0 (fwd_u, fwd_a hold those steps), and the
  // gradient on the nodal points once every step has run
  int run_exact(int64_t k0, int64_t k1);
  int finalize_exact();
  int check_status();
  bool tensor_core_path() const { return use_tc; }
  // doubles per step and shot in a forward-field store, and where its boundary part starts:
  // every nodal point, or the boundary nodes alone for the comparison method (no radial interior)
  int64_t store_stride() const { return md.lfe ? N : np; }
  int64_t store_bnd_off() const { return md.lfe ? 0 : nint; }
  // the Newmark state between windows, as one flat array of state_doubles() values
  int64_t state_doubles() const;
  int save_state(double* dst);
  int restore_state(const double* src);
  // zero one shot column of the Newmark state (and of the gradient accumulators)
  int zero_column(int s);

 private:
  int nb = 0, n = 0;
  int64_t E = 0, N = 0, np = 0, nint = 0;
  bool use_tc = false, persistent = false;
  bool use_mixed = false;            // per-class kernels (one-tile tensor-core + FP64) on an uneven mesh
  DevBuf elems_tc, elems_fp;         // the element classes of the mixed kernels
  int64_t n_tc = 0, n_fp = 0;
  ElemStepArgs ea;
  SolveArgs sa;
  PersistentSolveArgs pa;
  BoundaryArgs ba;
  const Task* ftasks = nullptr;
  const Task* btasks = nullptr;
  size_t s_smem = 0, e_smem = 0;
  int e_threads = 0, p_grid = 0;
  unsigned e_blocks = 0, b_blocks = 0;
  DevBuf bar, pstatus;
  LevelTasks* lt = nullptr;
  bool flow = false;                 // dataflow solve (default) instead of level barriers
  DevBuf flow_counters;              // done_f [nodes] | done_b [nodes] | item counters (u64, one per launch segment)
  int flow_grid[3] = {0, 0, 0};      // blocks of each dataflow launch segment
  size_t flow_smem[3] = {0, 0, 0};   // and its staging area (bytes)
  FlowArgs fa;
  unsigned flow_gen = 0;
  ExactElemArgs xa;
  ExactBoundaryArgs xba;
  ExactGradArgs xga;
  bool use_window = false;
  cudaAccessPolicyWindow window = {};
  int setup_l2_window(int device);
  int launch_solve(const void* fn, unsigned grid, void** args, bool cooperative, size_t smem = 0);
  std::vector<DevBuf*> state_bufs() const;
  int element_launch(int down, int up, int64_t done_step);
  int solve();
};

int Stepper::init() {
  const Mesh& m = *md.mesh;
  const Tree& t = m.tree;
  nb = md.nb; n = md.n;
  E = md.E; N = md.N; np = m.n_nodal; nint = m.n_int;
  // boundary state has one extra zero row: the padding dofs of uneven meshes read it
  const int64_t si = nint * B, sb = N * B, sb1 = (N + 1) * B;
  // element kernel: FP16 tensor cores with error-free splitting when the shapes allow,
  // else FP64 (SBFWI_ELEMENT=fp64 forces the FP64 kernel)
  const char* elem_env = std::getenv("SBFWI_ELEMENT");
  const bool exact = md.grad_mode == SBFWI_GRAD_EXACT || mode == Mode::Exact;
  if (md.lfe) {
    use_tc = false;                  // the comparison method has no radial interior
    if (mode == Mode::Exact) return fail(SBFWI_EUNSUPPORTED, "the exact adjoint is not built for the comparison method");
  } else if (exact) {
    // the exact adjoint keeps u and u'' of every step, which the FP64 kernel writes
    if (md.elem_pref == SBFWI_ELEMENT_TENSOR)
      return fail(SBFWI_EUNSUPPORTED, "the exact adjoint runs the FP64 element kernel, not the tensor-core one");
    use_tc = false;
  } else if (md.elem_pref == SBFWI_ELEMENT_TENSOR) {
    if (!tc_available(nb, B))
      return fail(SBFWI_EUNSUPPORTED, "no tensor-core element kernel for this n_b and shot count");
    use_tc = true;
  } else if (md.elem_pref == SBFWI_ELEMENT_FP64) {
    use_tc = false;
  } else if (md.elem_pref == SBFWI_ELEMENT_MIXED) {
    use_tc = false;
    use_mixed = true;
  } else {
    use_tc = tc_supported(nb, B) && !(elem_env && std::strcmp(elem_env, "fp64") == 0);
  }
  // elements of one mesh with different n_b: those with n_b <= 16 on the one-tile tensor-core
  // kernel, the others on the FP64 kernel, each element keeping its own kernel's state
  int64_t n_small = 0;
  for (int32_t v : m.nbe) n_small += v <= 16 ? 1 : 0;
  const bool mixed_ok = !md.lfe && !exact && B <= 8 && nb > 16 && n_small > 0 && n_small < E;
  if (use_mixed && !mixed_ok)
    return fail(SBFWI_EUNSUPPORTED, "mixed element kernels need elements on both sides of n_b = 16 and at most 8 shots");
  if (md.elem_pref == SBFWI_ELEMENT_AUTO && mixed_ok && !tc_supported(nb, B) &&
      !(elem_env && std::strcmp(elem_env, "fp64") == 0))
    use_mixed = true;                // padded n_b 17..20 or beyond 32
  if (use_tc && (!md.tc_ready || md.tc_one_tile)) {
    const int rc_tc = tc_prepare(md, st);
    if (rc_tc) return rc_tc;
  }
  if (use_mixed) {
    if (!md.tc_ready || !md.tc_one_tile) {
      const int rc_tc = tc_prepare_one_tile(md, st);
      if (rc_tc) return rc_tc;
    }
    std::vector<int32_t> small, large;
    for (int64_t e = 0; e < E; ++e) (m.nbe[e] <= 16 ? small : large).push_back((int32_t)e);
    SBFWI_CUDA(elems_tc.alloc(sizeof(int32_t) * small.size()));
    SBFWI_CUDA(elems_fp.alloc(sizeof(int32_t) * large.size()));
    SBFWI_CUDA(cudaMemcpy(elems_tc.p, small.data(), sizeof(int32_t) * small.size(), cudaMemcpyHostToDevice));
    SBFWI_CUDA(cudaMemcpy(elems_fp.p, large.data(), sizeof(int32_t) * large.size(), cudaMemcpyHostToDevice));
    n_tc = (int64_t)small.size();
    n_fp = (int64_t)large.size();
  }
  // the tensor-core path carries the predictor v and z = u' + dt (1 - gamma) u'' (in ud), not u, u''
  // the comparison method keeps no interior state
  const int64_t si_state = md.lfe ? 1 : si;
  SBFWI_CUDA(rb.u.alloc(sizeof(double) * (use_tc ? 1 : si_state)));
  SBFWI_CUDA(rb.ud.alloc(sizeof(double) * si_state));
  SBFWI_CUDA(rb.udd.alloc(sizeof(double) * (use_tc ? 1 : si_state)));
  SBFWI_CUDA(rb.q.alloc(sizeof(double) * si_state));
  if (use_tc || use_mixed) SBFWI_CUDA(rb.v.alloc(sizeof(double) * si));
  SBFWI_CUDA(rb.ub.alloc(sizeof(double) * sb1));
  SBFWI_CUDA(rb.udb.alloc(sizeof(double) * sb1));
  SBFWI_CUDA(rb.uddb.alloc(sizeof(double) * sb1));
  SBFWI_CUDA(rb.ext.alloc(sizeof(double) * sb));
  SBFWI_CUDA(rb.x.alloc(sizeof(double) * sb));
  SBFWI_CUDA(rb.fhat.alloc(sizeof(double) * E * nb * B));
  SBFWI_CUDA(rb.ysep.alloc(sizeof(double) * std::max<int64_t>(t.sep_rows, 1) * B));
  SBFWI_CUDA(rb.ybnd.alloc(sizeof(double) * std::max<int64_t>(t.bnd_rows, 1) * B));
  if (mode == Mode::Adjoint) {
    SBFWI_CUDA(rb.grad_int.alloc(sizeof(double) * np * B));
    SBFWI_CUDA(cudaMemsetAsync(rb.grad_int.p, 0, rb.grad_int.bytes, st));
  }
  if (mode == Mode::Exact) {
    int rc_x = prepare_exact(md, st);
    if (rc_x) return rc_x;
    const int ng = (3 * m.p + 2) / 2;
    SBFWI_CUDA(rb.mu.alloc(sizeof(double) * E * (n + 2) * nb * B));
    SBFWI_CUDA(rb.vbn.alloc(sizeof(double) * E * nb * B));
    SBFWI_CUDA(rb.ghost.alloc(sizeof(double) * E * 2 * nb * B));
    SBFWI_CUDA(rb.gacc.alloc(sizeof(double) * E * (n + 1) * 4 * m.L * ng));
    SBFWI_CUDA(rb.gbnd.alloc(sizeof(double) * E * nb));
    SBFWI_CUDA(rb.grad_int.alloc(sizeof(double) * np));
    for (DevBuf* b : {&rb.mu, &rb.vbn, &rb.ghost, &rb.gacc, &rb.gbnd, &rb.grad_int})
      SBFWI_CUDA(cudaMemsetAsync(b->p, 0, b->bytes, st));
  }
  int rc = zero_state();
  if (rc) return rc;
  // the solve's tasks are built for 4 blocks per SM; a block task stages its front's
  // vectors and its rows of the factors in shared memory, a warp task the same for a
  // whole small front, one slice per warp
  int device = 0, coop = 0, sms = 0, per_sm = 0;
  SBFWI_CUDA(cudaGetDevice(&device));
  SBFWI_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
  SBFWI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int grid = 4 * sms;
  lt = tasks_own ? tasks_own : &md.tasks;
  if (lt->shots != B || lt->grid != grid) {
    rc = build_level_tasks(md, *lt, B, grid);
    if (rc) return rc;
  }
  s_smem = sizeof(double) * std::max(lt->block_doubles, 8 * solve_warp_doubles(B));
  if (s_smem > 200 * 1024) return fail(SBFWI_EUNSUPPORTED, "solve staging area exceeds shared memory");
  for (const void* f : {(const void*)solve_forward_kernel, (const void*)solve_backward_kernel,
                        (const void*)solve_persistent_kernel, (const void*)solve_flow_kernel<false>,
                        (const void*)solve_flow_kernel<true>})
    if (s_smem > 48 * 1024) SBFWI_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_smem));

  ea.nb = nb; ea.n = n; ea.B = B; ea.E = E;
  ea.epc = std::max(1, 128 / (nb * B));
  ea.a0 = md.a0; ea.a1 = md.a1; ea.a2 = md.a2; ea.c1 = md.c1; ea.c2 = md.c2; ea.dt = md.dt;
  ea.mats = md.mats.as<double>(); ea.rt = md.rt.as<double>(); ea.dofs = md.dev().dofs.as<int32_t>();
  ea.u = rb.u.as<double>(); ea.ud = rb.ud.as<double>(); ea.udd = rb.udd.as<double>();
  ea.ub = rb.ub.as<double>(); ea.udb = rb.udb.as<double>(); ea.uddb = rb.uddb.as<double>();
  ea.q = rb.q.as<double>(); ea.fhat = rb.fhat.as<double>();
  ea.u_out = nullptr; ea.a_out = nullptr;
  if (mode == Mode::Adjoint && md.kernel_terms == SBFWI_TERMS_FULL) {
    SBFWI_CUDA(rb.lam.alloc(sizeof(double) * std::max<int64_t>(si, 1)));
    SBFWI_CUDA(cudaMemsetAsync(rb.lam.p, 0, rb.lam.bytes, st));
    int rc_g = ensure_gradient_operator(*md.mesh, st);
    if (rc_g) return rc_g;
  }
  e_threads = ea.epc * nb * B;
  ea.elems = use_mixed ? elems_fp.as<int32_t>() : nullptr;
  ea.n_elems = use_mixed ? n_fp : E;
  e_blocks = (unsigned)std::max<int64_t>(1, (ea.n_elems + ea.epc - 1) / ea.epc);
  e_smem = sizeof(double) * (size_t)ea.epc * (n + 2) * nb * B;
  cudaFuncAttributes eattr;
  SBFWI_CUDA(cudaFuncGetAttributes(&eattr, element_step_kernel));
  if (!use_tc && !md.lfe && (e_threads > eattr.maxThreadsPerBlock || e_smem > 227 * 1024))
    return fail(SBFWI_EUNSUPPORTED, "n_b x shots x radial points too large for one element block: run fewer shots per pass");
  if (e_smem > 48 * 1024 && !md.lfe)
    SBFWI_CUDA(cudaFuncSetAttribute(element_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e_smem));

  const MeshDevice& mdev = md.dev();
  sa.sep_nodes = md.solve_sep; sa.bnd_nodes = md.solve_bnd;
  sa.src0 = md.solve_src0; sa.src1 = md.solve_src1;
  // the exact adjoint solves with the transposed matrix: same tree, transposed factors
  sa.factors = mode == Mode::Exact ? md.factors_t.as<double>() : md.factors.as<double>();
  sa.fhat = rb.fhat.as<double>(); sa.ext = rb.ext.as<double>();
  sa.ysep = rb.ysep.as<double>(); sa.ybnd = rb.ybnd.as<double>(); sa.x = rb.x.as<double>();
  sa.nb = nb; sa.B = B;
  sa.warp_doubles = (int)solve_warp_doubles(B);
  sa.bdiv = B >= 2 ? (unsigned)((1ULL << 32) / (unsigned long long)B + 1ULL) : 0u;

  // one cooperative persistent launch per time step for the whole tree, unless the
  // device cannot launch cooperatively or SBFWI_SOLVE=levels asks for one launch per level
  SBFWI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_persistent_kernel, 256, s_smem));
  // SBFWI_SOLVE=levels: one launch per tree level; =barrier: one launch with grid
  // barriers between levels; default: one dataflow launch
  const char* solve_env = std::getenv("SBFWI_SOLVE");
  const bool can_coop = coop && per_sm > 0;
  if (md.solve_pref == SBFWI_SOLVE_AUTO) {
    persistent = can_coop && !(solve_env && std::strcmp(solve_env, "levels") == 0);
    flow = persistent && !(solve_env && std::strcmp(solve_env, "barrier") == 0);
  } else {
    if (md.solve_pref != SBFWI_SOLVE_LEVELS && !can_coop)
      return fail(SBFWI_EUNSUPPORTED, "this device cannot launch the cooperative solve schedules");
    persistent = md.solve_pref != SBFWI_SOLVE_LEVELS;
    flow = md.solve_pref == SBFWI_SOLVE_DATAFLOW;
  }
  ftasks = lt->fwd.as<Task>();
  btasks = lt->bwd.as<Task>();
  rc = mode == Mode::Exact ? SBFWI_OK : setup_l2_window(device);   // the window covers the forward factors
  if (rc) return rc;
  // status word of the bounded device waits (the solve's barriers and counters, the element
  // kernels' copy barriers)
  SBFWI_CUDA(pstatus.alloc(sizeof(int)));
  SBFWI_CUDA(cudaMemsetAsync(pstatus.p, 0, pstatus.bytes, st));
  if (persistent) {
    SBFWI_CUDA(bar.alloc(2 * sizeof(unsigned)));
    SBFWI_CUDA(cudaMemsetAsync(bar.p, 0, bar.bytes, st));
    pa.s = sa;
    pa.fwd = ftasks; pa.bwd = btasks;
    pa.fwd_meta = lt->fwd_meta.as<int32_t>(); pa.bwd_meta = lt->bwd_meta.as<int32_t>();
    pa.levels = t.levels;
    pa.bar = bar.as<unsigned>(); pa.status = pstatus.as<int>();
    pa.budget = 4000000000LL;            // ~2 s at 2 GHz
    pa.trace = nullptr;
    p_grid = std::max(1, std::min(std::min(per_sm, 4) * sms, lt->max_level_items));
  }
  if (flow) {
    // segment 1 (upper levels) stages up to s_smem, segments 0 and 2 the warp tasks' area
    const size_t small = std::min(s_smem, sizeof(double) * lt->small_doubles);
    flow_smem[0] = flow_smem[2] = small;
    flow_smem[1] = s_smem;
    for (int g = 0; g < 3; ++g) {
      int per_sm_flow = 0;
      SBFWI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_flow, solve_flow_kernel<true>, 256, flow_smem[g]));
      if (per_sm_flow < 1) return fail(SBFWI_EUNSUPPORTED, "the dataflow solve does not fit on an SM");
      flow_grid[g] = std::max(1, std::min(per_sm_flow, 4) * sms);   // every block co-resident (cooperative launch)
    }
    const int T = lt->nodes;
    const size_t cb = ((sizeof(unsigned) * 2 * (size_t)T + 15) / 16) * 16;
    SBFWI_CUDA(flow_counters.alloc(cb + 3 * sizeof(unsigned long long)));
    SBFWI_CUDA(cudaMemsetAsync(flow_counters.p, 0, flow_counters.bytes, st));
    fa.s = sa;
    fa.fwd = ftasks; fa.bwd = btasks;
    fa.items = lt->flow_items.as<int4>(); fa.n_items = lt->n_items;
    fa.node_info = lt->node_info.as<int32_t>(); fa.nodes = T;
    fa.done_f = flow_counters.as<unsigned>(); fa.done_b = fa.done_f + T;
    fa.claim = reinterpret_cast<unsigned long long*>(flow_counters.as<char>() + cb);
    fa.status = pstatus.as<int>();
    fa.budget = 4000000000LL;
    fa.levels = md.mesh->tree.levels;
    fa.trace = nullptr;
    p_grid = flow_grid[0];
    flow_gen = 0;
  }

  ba.N = N; ba.B = B; ba.R = 0;
  ba.K = K;
  ba.a0 = md.a0; ba.a1 = md.a1; ba.a2 = md.a2; ba.c1 = md.c1; ba.c2 = md.c2; ba.dt = md.dt;
  ba.x = rb.x.as<double>(); ba.ub = rb.ub.as<double>(); ba.udb = rb.udb.as<double>(); ba.uddb = rb.uddb.as<double>();
  ba.rec = nullptr; ba.traces = nullptr; ba.store_b = nullptr; ba.store_ub = nullptr; ba.store_ab = nullptr;
  ba.fwd_b = nullptr; ba.grad_b = nullptr;
  b_blocks = (unsigned)std::min<int64_t>((sb + 255) / 256, 152 * 8);

  if (mode == Mode::Exact) {
    const double beta = md.beta, gamma = md.gamma, dt = md.dt;
    xa.nb = nb; xa.n = n; xa.B = B; xa.E = E; xa.N = N;
    xa.epc = std::max(1, 128 / (nb * B));
    xa.a0 = md.a0; xa.a1 = md.a1; xa.a2 = md.a2;
    xa.cu = gamma / (beta * dt); xa.cud = 1.0 - gamma / beta; xa.cudd = dt * (1.0 - gamma / (2.0 * beta));
    xa.du = 1.0 / (beta * dt * dt); xa.dud = -1.0 / (beta * dt); xa.dudd = 1.0 - 1.0 / (2.0 * beta);
    xa.mats = md.mats.as<double>(); xa.rt = md.rt.as<double>();
    xa.xops = md.xops.as<double>(); xa.xel = md.xel.as<double>(); xa.dofs = md.dev().dofs.as<int32_t>();
    xa.ua = rb.u.as<double>(); xa.uda = rb.ud.as<double>(); xa.udda = rb.udd.as<double>();
    xa.s = rb.q.as<double>(); xa.fbar = rb.x.as<double>(); xa.mu = rb.mu.as<double>(); xa.vbn = rb.vbn.as<double>();
    xa.fhat = rb.fhat.as<double>(); xa.ghost = rb.ghost.as<double>();
    xa.fu_int = xa.fu_b = xa.fa_b = nullptr;
    if (xa.epc * nb * B > 512 || exact_element_smem(nb, n, B, xa.epc) > 227 * 1024)
      return fail(SBFWI_EUNSUPPORTED, "n_b x shots x radial points too large for one element block of the exact adjoint");
    xba.N = N; xba.B = B;
    xba.a0 = md.a0; xba.a1 = md.a1; xba.a2 = md.a2;
    xba.cu = xa.cu; xba.cud = xa.cud; xba.cudd = xa.cudd; xba.du = xa.du; xba.dud = xa.dud; xba.dudd = xa.dudd;
    xba.ub = rb.ub.as<double>(); xba.udb = rb.udb.as<double>(); xba.uddb = rb.uddb.as<double>();
    xba.ext = rb.ext.as<double>(); xba.vbn = rb.vbn.as<double>();
    xba.inc_ptr = md.dev().inc_ptr.as<int64_t>(); xba.inc_list = md.dev().inc_list.as<int64_t>();
    int Bp = 1;
    while (Bp < B) Bp <<= 1;
    xga.E = E; xga.N = N; xga.nb = nb; xga.n = n; xga.B = B; xga.Bp = Bp; xga.L = m.L; xga.ng = (3 * m.p + 2) / 2;
    xga.h = (1.0 - m.xi0) / n;
    xga.xi = md.dev().xih.as<double>(); xga.tab = md.dev().tab.as<double>();
    xga.lptr = md.dev().lptr.as<int64_t>(); xga.line_local = md.dev().lloc.as<int32_t>();
    xga.dofs = md.dev().dofs.as<int32_t>();
    xga.mu = rb.mu.as<double>(); xga.fbar = rb.x.as<double>(); xga.ghost = rb.ghost.as<double>();
    xga.gacc = rb.gacc.as<double>();
  }
  return SBFWI_OK;
}

// The solve reads the same factors and index arrays every step, but the element
// kernel streams gigabytes through L2 in between and would evict them.  Mark that one
// range persisting (an access policy window on the solve launches) and, if the
// context's persisting L2 set-aside is smaller, raise it to cover the range (a limit
// of this process's context; SBFWI_L2_PERSIST=0 leaves L2 alone).
int Stepper::setup_l2_window(int device) {
  use_window = false;
  const char* env = std::getenv("SBFWI_L2_PERSIST");
  if (env && std::strcmp(env, "0") == 0) return SBFWI_OK;
  int max_persist = 0, max_window = 0;
  if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, device) != cudaSuccess) {
    cudaGetLastError();
    return SBFWI_OK;
  }
  if (max_persist <= 0 || max_window <= 0 || md.solve_bytes == 0) return SBFWI_OK;
  const size_t want = std::min(md.solve_bytes, (size_t)max_persist);
  size_t cur = 0;
  SBFWI_CUDA(cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
  if (cur < want) {
    SBFWI_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
    SBFWI_CUDA(cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
  }
  if (cur == 0) return SBFWI_OK;
  window.base_ptr = md.factors.p;
  window.num_bytes = std::min(md.solve_bytes, (size_t)max_window);
  window.hitRatio = (float)std::min(1.0, (double)cur / (double)window.num_bytes);
  window.hitProp = cudaAccessPropertyPersisting;
  window.missProp = cudaAccessPropertyStreaming;
  use_window = true;
  return SBFWI_OK;
}

int Stepper::launch_solve(const void* fn, unsigned grid, void** args, bool cooperative, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem ? smem : s_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (cooperative) {
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
  }
  if (use_window) {
    attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[na].val.accessPolicyWindow = window;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  SBFWI_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
  return SBFWI_OK;
}

int Stepper::zero_state() {
  for (DevBuf* b : {&rb.u, &rb.ud, &rb.udd, &rb.v, &rb.q, &rb.ub, &rb.udb, &rb.uddb, &rb.ext, &rb.x, &rb.fhat})
    if (b->p) SBFWI_CUDA(cudaMemsetAsync(b->p, 0, b->bytes, st));
  return SBFWI_OK;
}

std::vector<DevBuf*> Stepper::state_bufs() const {
  if (use_tc) return {&rb.v, &rb.ud, &rb.ub, &rb.udb, &rb.uddb};
  if (use_mixed) return {&rb.u, &rb.ud, &rb.udd, &rb.v, &rb.ub, &rb.udb, &rb.uddb};
  return {&rb.u, &rb.ud, &rb.udd, &rb.ub, &rb.udb, &rb.uddb};
}

int64_t Stepper::state_doubles() const {
  int64_t tot = 0;
  for (DevBuf* b : state_bufs()) tot += (int64_t)(b->bytes / sizeof(double));
  return tot;
}

int Stepper::save_state(double* dst) {
  for (DevBuf* b : state_bufs()) {
    SBFWI_CUDA(cudaMemcpyAsync(dst, b->p, b->bytes, cudaMemcpyDeviceToDevice, st));
    dst += b->bytes / sizeof(double);
  }
  return SBFWI_OK;
}

int Stepper::restore_state(const double* src) {
  int rc = zero_state();
  if (rc) return rc;
  for (DevBuf* b : state_bufs()) {
    SBFWI_CUDA(cudaMemcpyAsync(b->p, src, b->bytes, cudaMemcpyDeviceToDevice, st));
    src += b->bytes / sizeof(double);
  }
  return SBFWI_OK;
}

int Stepper::element_launch(int down, int up, int64_t done_step) {
  // done_step: the step whose back-substitution runs in this launch (if down)
  Profiler& prof = profiler();
  if (md.lfe) {                      // comparison method: only the effective sources of the next step
    if (up) {
      prof.begin(kPhaseElement, st);
      const int64_t tot = E * nb * B;
      const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16);
      lfe_source_kernel<<<blocks, 256, 0, st>>>(md.lfe_M.as<double>(), md.dev().dofs.as<int32_t>(), rb.ub.as<double>(),
                                                 rb.udb.as<double>(), rb.uddb.as<double>(), E, nb, B, md.a0, md.a1,
                                                 md.a2, rb.fhat.as<double>());
      prof.end(kPhaseElement, st);
      prof.count(kPhaseElement);
    }
    return SBFWI_OK;
  }
  ea.do_down = down; ea.do_up = up;
  ea.store_int = nullptr; ea.fwd_int = nullptr; ea.grad_int = nullptr; ea.u_out = nullptr;
  if (down && mode == Mode::Forward && store) ea.store_int = store + (done_step - store_k0) * np * B;
  if (down && mode == Mode::Forward && store_u) ea.u_out = store_u + (done_step - store_k0) * np * B;
  ea.a_out = (down && mode == Mode::Forward && store_a) ? store_a + (done_step - store_k0) * np * B : nullptr;
  const bool grad_term = down && mode == Mode::Adjoint && fwd_u != nullptr;
  if (grad_term) ea.u_out = rb.lam.as<double>();
  if (down && mode == Mode::Adjoint) {
    ea.fwd_int = fwd + (K - 1 - done_step - fwd_k0) * np * B;
    ea.grad_int = rb.grad_int.as<double>();
  }
  prof.begin(kPhaseElement, st);
  if (use_tc || use_mixed)
    tc_element_launch(md, B, down, up, ea.u, ea.ud, ea.udd, rb.v.as<double>(), ea.ub, ea.udb, ea.uddb, ea.q, ea.fhat,
                      ea.store_int, ea.fwd_int, ea.grad_int, ea.u_out, st, use_mixed ? elems_tc.as<int32_t>() : nullptr,
                      n_tc, pstatus.as<int>());
  if (!use_tc && (!use_mixed || n_fp > 0)) element_step_kernel<<<e_blocks, e_threads, e_smem, st>>>(ea);
  prof.end(kPhaseElement, st);
  prof.count(kPhaseElement, use_mixed ? 2 : 1);
  if (grad_term) {
    // the full kernel's gradient term of this step: the interior adjoint field was just
    // written to lam, its boundary part is the current boundary state
    const MeshDevice& mdev = md.dev();
    const int64_t tot = np * B;
    const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16);
    gradient_term_kernel<<<blocks, 256, 0, st>>>(mdev.grad_ptr.as<int64_t>(), mdev.grad_col.as<int32_t>(),
                                                 mdev.grad_val.as<double>(), np, nint, B,
                                                 fwd_u + (K - 1 - done_step - fwd_k0) * np * B, rb.lam.as<double>(),
                                                 rb.ub.as<double>(), md.c * md.c, rb.grad_int.as<double>());
    prof.count(kPhaseOther);
  }
  return SBFWI_OK;
}

int Stepper::solve() {
  Profiler& prof = profiler();
  const Tree& t = md.mesh->tree;
  prof.begin(kPhaseSolve, st);
  if (flow) {
    ++flow_gen;
    unsigned long long* trace = prof.flow_trace(2 * t.levels, st);
    // up to three launches in stream order (lower forward levels, upper levels, lower backward
    // levels), each claiming its own range of the topologically ordered items
    for (int g = 0; g < 3; ++g) {
      const int i0 = lt->flow_seg[g], i1 = lt->flow_seg[g + 1];
      if (i1 <= i0) continue;
      FlowArgs f = fa;
      f.gen = flow_gen;
      f.trace = trace;
      f.items = lt->flow_items.as<int4>() + i0;
      f.n_items = i1 - i0;
      f.claim = fa.claim + g;
      f.base = (unsigned long long)(flow_gen - 1) * (unsigned long long)(f.n_items + flow_grid[g]);
      void* kargs[] = {&f};
      int rc = launch_solve(trace ? (const void*)solve_flow_kernel<true> : (const void*)solve_flow_kernel<false>,
                            (unsigned)flow_grid[g], kargs, true, flow_smem[g]);
      if (rc) return rc;
      prof.count(kPhaseSolve);
    }
  } else if (persistent) {
    pa.trace = prof.level_trace(6 * t.levels, st);
    if (pa.trace) ++prof.level_steps;
    void* kargs[] = {&pa};
    int rc = launch_solve((const void*)solve_persistent_kernel, (unsigned)p_grid, kargs, true);
    if (rc) return rc;
    prof.count(kPhaseSolve);
  } else {
    LevelKernelArgs la;
    la.s = sa; la.levels = t.levels;
    for (int l = 0; l < t.levels; ++l) {
      const int cnt = lt->items(true, l);
      if (cnt == 0) continue;
      la.tasks = ftasks; la.meta = lt->fwd_meta.as<int32_t>(); la.level = l;
      void* kargs[] = {&la};
      int rc = launch_solve((const void*)solve_forward_kernel, (unsigned)cnt, kargs, false);
      if (rc) return rc;
      prof.count(kPhaseSolve);
    }
    for (int l = t.levels - 1; l >= 0; --l) {
      const int cnt = lt->items(false, l);
      if (cnt == 0) continue;
      la.tasks = btasks; la.meta = lt->bwd_meta.as<int32_t>(); la.level = l;
      void* kargs[] = {&la};
      int rc = launch_solve((const void*)solve_backward_kernel, (unsigned)cnt, kargs, false);
      if (rc) return rc;
      prof.count(kPhaseSolve);
    }
  }
  prof.end(kPhaseSolve, st);
  return SBFWI_OK;
}

int Stepper::run(int64_t k0, int64_t k1) {
  Profiler& prof = profiler();
  if (k0 < 0 || k1 > K || k0 >= k1) return fail(SBFWI_EINVAL, "bad step window");
  // the forward sweep of step k0 (at k0 = 0 the zero state gives f_hat = 0, unless resuming)
  if (k0 > 0 || resume) element_launch(0, 1, k0 - 1);
  for (int64_t k = k0; k < k1; ++k) {
    if (k > k0) element_launch(1, 1, k - 1);
    // sources of step k
    if (mode == Mode::Forward) {
      sources_kernel<<<(B + 127) / 128, 128, 0, st>>>(rb.ext.as<double>(), B, 1, nodes, values, K, k, 1);
      prof.count(kPhaseOther);
    } else if (R > 0) {
      sources_kernel<<<(B * R + 127) / 128, 128, 0, st>>>(rb.ext.as<double>(), B, R, nodes, values, K, K - 1 - k, 0);
      prof.count(kPhaseOther);
    }
    int rc = solve();
    if (rc) return rc;
    ba.k = k;
    if (mode == Mode::Forward) {
      ba.R = R;
      ba.rec = nodes + B;
      ba.traces = R > 0 ? traces : nullptr;
      ba.store_b = store ? store + ((k - store_k0) * store_stride() + store_bnd_off()) * B : nullptr;
      ba.store_ub = store_u ? store_u + (k - store_k0) * np * B + nint * B : nullptr;
      ba.store_ab = store_a ? store_a + (k - store_k0) * np * B + nint * B : nullptr;
    } else {
      ba.fwd_b = fwd + ((K - 1 - k - fwd_k0) * store_stride() + store_bnd_off()) * B;
      ba.grad_b = rb.grad_int.as<double>() + nint * B;
    }
    boundary_update_kernel<<<b_blocks, 256, 0, st>>>(ba);
    prof.count(kPhaseOther);
  }
  element_launch(1, 0, k1 - 1);
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

int Stepper::run_exact(int64_t k0, int64_t k1) {
  Profiler& prof = profiler();
  if (mode != Mode::Exact) return fail(SBFWI_ESTATE, "not an exact-adjoint stepper");
  if (k0 < 0 || k1 > K || k0 >= k1) return fail(SBFWI_EINVAL, "bad step window");
  int rc;
  for (int64_t k = k1 - 1; k >= k0; --k) {
    // the misfit's share at the receivers, then x_bar of the boundary nodes
    if ((rc = exact_misfit_launch(rb.ub.as<double>(), B, R, nodes, values, K, k, md.dt, st))) return rc;
    if ((rc = exact_boundary_launch(xba, false, st))) return rc;
    prof.count(kPhaseOther, R > 0 ? 2 : 1);
    if ((rc = solve())) return rc;
    // the forward solution after step k
    const double* fu = fwd_u + (k - fwd_k0) * np * B;
    const double* fa_ = fwd_a + (k - fwd_k0) * np * B;
    xa.fu_int = fu; xa.fu_b = fu + nint * B; xa.fa_b = fa_ + nint * B;
    xa.do_down = 1; xa.do_up = k > 0 ? 1 : 0;
    prof.begin(kPhaseElement, st);
    rc = exact_element_launch(xa, st);
    prof.end(kPhaseElement, st);
    prof.count(kPhaseElement);
    if (rc) return rc;
    if ((rc = exact_boundary_launch(xba, true, st))) return rc;
    xga.fu_int = fu; xga.fu_b = fu + nint * B; xga.fa_int = fa_; xga.fa_b = fa_ + nint * B;
    if ((rc = exact_gradient_launch(xga, md.mesh->p, st))) return rc;
    prof.count(kPhaseOther, 2);
  }
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

int Stepper::finalize_exact() {
  const Mesh& m = *md.mesh;
  ExactFinalArgs f;
  f.E = E; f.nb = nb; f.n = n; f.pp = m.p + 1; f.ng = (3 * m.p + 2) / 2; f.L = m.L;
  f.lptr = md.dev().lptr.as<int64_t>(); f.line_local = md.dev().lloc.as<int32_t>(); f.tab = md.dev().tab.as<double>();
  f.kq = md.kq.as<double>(); f.gacc = rb.gacc.as<double>();
  f.g_nodal = rb.grad_int.as<double>(); f.g_bnd = rb.gbnd.as<double>();
  int rc = exact_finalize_launch(f, md.dev().inc_ptr.as<int64_t>(), md.dev().inc_list.as<int64_t>(), N,
                                 rb.grad_int.as<double>() + nint, st);
  profiler().count(kPhaseOther, 2);
  return rc;
}

int Stepper::check_status() {
  int code = 0;
  SBFWI_CUDA(cudaMemcpyAsync(&code, pstatus.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SBFWI_CUDA(cudaStreamSynchronize(st));
  if (code) return fail(SBFWI_ETIMEOUT, "a bounded device wait (global solve or element-kernel copy) timed out");
  return SBFWI_OK;
}

bool have_device() {
  int count = 0;
  return cudaGetDeviceCount(&count) == cudaSuccess && count > 0;
}

// ---------------------------------------------------------------------------
// sessions: continuous batching.  The shots of a session are the columns ("slots") of
// one resumable stepper; each slot carries its own request, admitted at a window boundary
// with a zero state and its own step offset, and retired when its steps are done.  A
// window runs W steps of every slot; the sources, traces and forward fields of the
// window pass through window buffers that kernels fill from, and empty into, each
// slot's own arrays at its own local step.
// ---------------------------------------------------------------------------
struct SlotDev {
  const double* values;   // forward: wavelet [K]; adjoint: residual [R][K]
  double* traces;         // forward: [R][K]
  double* field;          // forward: velocities [K][stride] out (nullable); adjoint: the forward ones in
  int64_t start, K;       // global step of the slot's first step, its step count
  int32_t active, pad;
};

__global__ void session_sources_kernel(const SlotDev* slots, int B, int R, int64_t k0, int W, int adjoint,
                                       double* out) {
  const int64_t tot = adjoint ? (int64_t)B * R * W : (int64_t)B * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % W);
    const int64_t sr = t / W;                       // forward: slot; adjoint: slot * R + receiver
    const int s = (int)(adjoint ? sr / R : sr);
    const SlotDev sl = slots[s];
    const int64_t m = k0 + j - sl.start;            // the slot's own step
    const bool in = sl.active && m >= 0 && m < sl.K;
    if (!adjoint) {
      out[t] = in ? sl.values[m] : 0.0;
    } else {
      // the window's adjoint step j injects the residual sample K - 1 - m, stored reversed as
      // the stepper reads it (column W - 1 - j of a window of W steps)
      const int r = (int)(sr - (int64_t)s * R);
      out[sr * W + (W - 1 - j)] = in ? sl.values[(int64_t)r * sl.K + (sl.K - 1 - m)] : 0.0;
    }
  }
}

__global__ void session_traces_kernel(const SlotDev* slots, int B, int R, int64_t k0, int W, const double* win) {
  const int64_t tot = (int64_t)B * R * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % W);
    const int64_t sr = t / W;
    const int s = (int)(sr / R), r = (int)(sr - (int64_t)s * R);
    const SlotDev sl = slots[s];
    const int64_t m = k0 + j - sl.start;
    if (sl.active && m >= 0 && m < sl.K) sl.traces[(int64_t)r * sl.K + m] = win[t];
  }
}

// forward: the window's nodal velocities [W][stride][B] go to each slot's field at its own
// step; adjoint: each slot's forward velocities are gathered into the window, reversed in
// time as the adjoint stepper pairs them
__global__ void session_field_kernel(const SlotDev* slots, int B, int64_t stride, int64_t k0, int W, int adjoint,
                                     double* win) {
  const int64_t tot = (int64_t)W * stride * B;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t % B);
    const int64_t jq = t / B;
    const int j = (int)(jq / stride);
    const int64_t q = jq - (int64_t)j * stride;
    const SlotDev sl = slots[s];
    const int64_t m = k0 + j - sl.start;
    const bool in = sl.active && sl.field && m >= 0 && m < sl.K;
    if (!adjoint) {
      if (in) sl.field[m * stride + q] = win[t];
    } else {
      win[((int64_t)(W - 1 - j) * stride + q) * B + s] = in ? sl.field[(sl.K - 1 - m) * stride + q] : 0.0;
    }
  }
}

__global__ void column_zero_kernel(double* buf, int64_t rows, int B, int s) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rows; q += (int64_t)gridDim.x * blockDim.x)
    buf[q * B + s] = 0.0;
}

__global__ void column_copy_kernel(const double* acc, int64_t rows, int B, int s, double scale, double* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rows; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = scale * acc[q * B + s];
}

int Stepper::zero_column(int s) {
  std::vector<DevBuf*> bufs = state_bufs();
  // the sources kernel writes only the column's current source node: the previous
  // request's last sample at its node must not act on the next one
  bufs.push_back(&rb.ext);
  if (mode == Mode::Adjoint) bufs.push_back(&rb.grad_int);
  for (DevBuf* b : bufs) {
    const int64_t rows = (int64_t)(b->bytes / sizeof(double)) / B;
    if (rows == 0) continue;
    column_zero_kernel<<<(unsigned)std::min<int64_t>((rows + 255) / 256, 152 * 8), 256, 0, st>>>(b->as<double>(), rows,
                                                                                                 B, s);
    profiler().count(kPhaseOther);
  }
  SBFWI_CUDA(cudaGetLastError());
  return SBFWI_OK;
}

struct SlotHost {
  bool active = false, finished = false;
  int64_t start = 0, K = 0;
  DevBuf values, traces;
  double* field = nullptr;
};

}  // namespace

// the gradient on the model's parameter layout from nodal values in the library's layout
static int emit_gradient(Model& md, const double* g_lib, double* grad, int mem, bool accumulate, cudaStream_t st);

struct Session {
  Model* md = nullptr;
  int kind = 0, B = 0, R = 0, W = 0;
  cudaStream_t st = nullptr;
  std::vector<int64_t> rec;
  RunBuffers rb;
  LevelTasks tasks;
  std::unique_ptr<Stepper> sp;
  DevBuf nodes, win_values, win_traces, win_field, slots_dev;
  std::vector<SlotHost> slots;
  std::vector<SlotDev> slots_h;
  int64_t kglob = 0;
  bool field_used = false;

  int upload_slots() {
    for (int s = 0; s < B; ++s) {
      const SlotHost& h = slots[s];
      SlotDev& d = slots_h[s];
      d.values = h.values.as<double>(); d.traces = h.traces.as<double>(); d.field = h.field;
      d.start = h.start; d.K = h.K; d.active = h.active ? 1 : 0; d.pad = 0;
    }
    SBFWI_CUDA(cudaMemcpyAsync(slots_dev.p, slots_h.data(), sizeof(SlotDev) * B, cudaMemcpyHostToDevice, st));
    // the host array must stay unchanged until the copy has run
    SBFWI_CUDA(cudaStreamSynchronize(st));
    return SBFWI_OK;
  }
};

}  // namespace sbfwi

struct sbfwi_session : public sbfwi::Session {};

namespace sbfwi {

static int emit_gradient(Model& md, const double* g_lib, double* grad, int mem, bool accumulate, cudaStream_t st) {
  const Mesh& msh = *md.mesh;
  const bool grid = md.rho_kind == SBFWI_RHO_GRID;
  const int64_t nout = grid ? md.gx * md.gy * (msh.dim == 3 ? md.gz : 1) : msh.n_nodal_api;
  DevBuf gout;
  double* dst = nullptr;
  if (mem == SBFWI_MEM_DEVICE) dst = grad;
  else {
    SBFWI_CUDA(gout.alloc(sizeof(double) * nout));
    dst = gout.as<double>();
    if (accumulate) SBFWI_CUDA(cudaMemcpyAsync(dst, grad, sizeof(double) * nout, cudaMemcpyHostToDevice, st));
  }
  const unsigned gb = (unsigned)std::min<int64_t>((nout + 255) / 256, 152 * 8);
  if (grid && msh.dim == 3) {
    // the transpose of the trilinear map of the fine grid
    const MeshDevice& mdev = md.dev();
    grid_transpose3d_kernel<<<gb, 256, 0, st>>>(g_lib, md.pts_hi.as<double>(), mdev.cell.as<int32_t>(),
                                                mdev.clamp.as<int8_t>(), mdev.cell_ptr.as<int64_t>(),
                                                mdev.cell_list.as<int64_t>(), md.gx, md.gy, md.gz, md.lx, md.ly,
                                                md.lz, dst, accumulate ? 1 : 0);
  } else if (grid) {
    // the transpose of the bilinear map of the fine grid
    const MeshDevice& mdev = md.dev();
    grid_transpose_kernel<<<gb, 256, 0, st>>>(g_lib, md.pts_hi.as<double>(), mdev.cell.as<int32_t>(),
                                              mdev.clamp.as<int8_t>(), mdev.cell_ptr.as<int64_t>(),
                                              mdev.cell_list.as<int64_t>(), md.gx, md.gy, md.lx, md.ly, dst,
                                              accumulate ? 1 : 0);
  } else if (msh.uneven) {
    // the padded layout gathered to the caller's
    gather_nodal_kernel<<<gb, 256, 0, st>>>(g_lib, md.dev().api_map.as<int64_t>(), nout, dst, accumulate ? 1 : 0);
  } else {
    sum_shots_kernel<<<gb, 256, 0, st>>>(g_lib, nout, 1, 1.0, dst, accumulate ? 1 : 0);
  }
  profiler().count(kPhaseOther);
  SBFWI_CUDA(cudaGetLastError());
  if (mem == SBFWI_MEM_HOST) SBFWI_CUDA(cudaMemcpyAsync(grad, dst, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
  SBFWI_CUDA(cudaStreamSynchronize(st));
  return SBFWI_OK;
}

}  // namespace sbfwi

using namespace sbfwi;

extern "C" {

static int set_model_impl(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho, int rho_kind,
                          int64_t gx, int64_t gy, int64_t gz, double lx, double ly, double lz, double dt, double beta,
                          double gamma, int mem, void* stream, bool lfe, int dim);

int sbfwi_set_model(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho, int rho_kind,
                    int64_t gx, int64_t gy, double lx, double ly, double dt, double beta, double gamma, int mem,
                    void* stream) {
  return set_model_impl(out, mesh, c, rho, rho_kind, gx, gy, 1, lx, ly, 1.0, dt, beta, gamma, mem, stream, false, 2);
}

int sbfwi_set_model_lfe(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho, int rho_kind,
                        int64_t gx, int64_t gy, double lx, double ly, double dt, double beta, double gamma, int mem,
                        void* stream) {
  return set_model_impl(out, mesh, c, rho, rho_kind, gx, gy, 1, lx, ly, 1.0, dt, beta, gamma, mem, stream, true, 2);
}

int sbfwi_set_model3d(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho, int rho_kind,
                      int64_t gx, int64_t gy, int64_t gz, double lx, double ly, double lz, double dt, double beta,
                      double gamma, int mem, void* stream) {
  if (rho_kind == SBFWI_RHO_GRID && (gz < 2 || !(lz > 0))) return fail(SBFWI_EINVAL, "grid density needs gz >= 2 and lz > 0");
  return set_model_impl(out, mesh, c, rho, rho_kind, gx, gy, gz, lx, ly, lz, dt, beta, gamma, mem, stream, false, 3);
}

static int set_model_impl(sbfwi_model** out, const sbfwi_mesh* mesh, double c, const double* rho, int rho_kind,
                          int64_t gx, int64_t gy, int64_t gz, double lx, double ly, double lz, double dt, double beta,
                          double gamma, int mem, void* stream, bool lfe, int dim) {
  if (!out) return fail(SBFWI_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !rho) return fail(SBFWI_EINVAL, "NULL argument");
  if (mesh->dim != dim)
    return fail(SBFWI_EINVAL, dim == 3 ? "sbfwi_set_model3d needs a mesh from sbfwi_build_mesh3d"
                                       : "a mesh from sbfwi_build_mesh3d needs sbfwi_set_model3d");
  if (!(c > 0) || !(dt > 0) || !(beta > 0) || !(gamma >= 0)) return fail(SBFWI_EINVAL, "need c > 0, dt > 0, beta > 0, gamma >= 0");
  if (rho_kind != SBFWI_RHO_GRID && rho_kind != SBFWI_RHO_NODAL) return fail(SBFWI_EINVAL, "unknown rho_kind");
  if (rho_kind == SBFWI_RHO_GRID && (gx < 2 || gy < 2 || !(lx > 0) || !(ly > 0)))
    return fail(SBFWI_EINVAL, "grid density needs gx, gy >= 2 and lx, ly > 0");
  if (mem != SBFWI_MEM_HOST && mem != SBFWI_MEM_DEVICE) return fail(SBFWI_EINVAL, "unknown mem");
  if (!have_device()) return fail(SBFWI_ECUDA, "no CUDA device");
  auto md = new sbfwi_model();
  md->mesh = mesh;
  md->c = c; md->dt = dt; md->beta = beta; md->gamma = gamma;
  md->a0 = 1.0 / (beta * dt * dt);
  md->a1 = 1.0 / (beta * dt);
  md->a2 = 1.0 / (2.0 * beta) - 1.0;
  md->c1 = dt * (1.0 - gamma);
  md->c2 = dt * gamma;
  md->rho_kind = rho_kind; md->gx = gx; md->gy = gy; md->gz = gz; md->lx = lx; md->ly = ly; md->lz = lz;
  md->lfe = lfe;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = setup_model(*md, *mesh, rho, mem, st);
  if (rc == SBFWI_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "set-up kernels");
  }
  profiler().resolve();
  if (rc != SBFWI_OK) { delete md; return rc; }
  *out = md;
  return SBFWI_OK;
}

void sbfwi_destroy_model(sbfwi_model* m) { delete m; }

int sbfwi_set_kernel_terms(sbfwi_model* m, int terms) {
  if (!m) return fail(SBFWI_EINVAL, "model is NULL");
  if (terms != SBFWI_TERMS_VELOCITY && terms != SBFWI_TERMS_FULL) return fail(SBFWI_EINVAL, "unknown kernel terms");
  if (terms == SBFWI_TERMS_FULL && m->mesh->dim == 3)
    return fail(SBFWI_EUNSUPPORTED, "the full kernel's gradient term is not built for 3-D meshes");
  m->kernel_terms = terms;
  return SBFWI_OK;
}

int sbfwi_set_gradient_mode(sbfwi_model* m, int mode) {
  if (!m) return fail(SBFWI_EINVAL, "model is NULL");
  if (mode != SBFWI_GRAD_KERNEL && mode != SBFWI_GRAD_EXACT) return fail(SBFWI_EINVAL, "unknown gradient mode");
  if (mode == SBFWI_GRAD_EXACT && m->lfe)
    return fail(SBFWI_EUNSUPPORTED, "the exact adjoint is not built for the comparison method");
  if (mode == SBFWI_GRAD_EXACT && m->mesh->dim == 3)
    return fail(SBFWI_EUNSUPPORTED, "the exact adjoint is not built for 3-D meshes");
  m->grad_mode = mode;
  return SBFWI_OK;
}

int sbfwi_set_schedule(sbfwi_model* m, int element, int solve) {
  if (!m) return fail(SBFWI_EINVAL, "model is NULL");
  if (element < SBFWI_ELEMENT_AUTO || element > SBFWI_ELEMENT_MIXED) return fail(SBFWI_EINVAL, "unknown element kernel");
  if (solve < SBFWI_SOLVE_AUTO || solve > SBFWI_SOLVE_LEVELS) return fail(SBFWI_EINVAL, "unknown solve schedule");
  m->elem_pref = element;
  m->solve_pref = solve;
  return SBFWI_OK;
}
void sbfwi_destroy_fwdstate(sbfwi_fwdstate* s) { delete s; }

int sbfwi_forward(sbfwi_model* md, int32_t n_shots, const int64_t* src_node, const double* src_wavelet, int32_t n_rec,
                  const int64_t* rec_node, int64_t K, double* traces, sbfwi_fwdstate** keep, int64_t ckpt_every,
                  int mem, void* stream) {
  if (keep) *keep = nullptr;
  if (!md) return fail(SBFWI_EINVAL, "model is NULL");
  if (n_shots < 1 || n_shots > kMaxShots) return fail(SBFWI_EINVAL, "n_shots must be in 1..16");
  if (K < 1) return fail(SBFWI_EINVAL, "K must be >= 1");
  if (n_rec < 0 || (n_rec > 0 && (!rec_node || !traces))) return fail(SBFWI_EINVAL, "receivers need rec_node and traces");
  if (!src_node || !src_wavelet) return fail(SBFWI_EINVAL, "NULL source arrays");
  if (mem != SBFWI_MEM_HOST && mem != SBFWI_MEM_DEVICE) return fail(SBFWI_EINVAL, "unknown mem");
  if (ckpt_every < SBFWI_CKPT_AUTO) return fail(SBFWI_EINVAL, "ckpt_every must be >= -1");
  const int64_t N = md->N;
  for (int s = 0; s < n_shots; ++s)
    if (src_node[s] < 0 || src_node[s] >= N) return fail(SBFWI_EINVAL, "source node out of range");
  for (int r = 0; r < n_rec; ++r) {
    if (rec_node[r] < 0 || rec_node[r] >= N) return fail(SBFWI_EINVAL, "receiver node out of range");
    for (int r2 = 0; r2 < r; ++r2)
      if (rec_node[r2] == rec_node[r]) return fail(SBFWI_EINVAL, "receiver nodes must be distinct");
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int B = n_shots;
  const int64_t np = md->mesh->n_nodal;
  DevBuf values, nodes, traces_owned;
  SBFWI_CUDA(values.alloc(sizeof(double) * B * K));
  SBFWI_CUDA(cudaMemcpyAsync(values.p, src_wavelet, sizeof(double) * B * K,
                             mem == SBFWI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  std::vector<int64_t> nv(src_node, src_node + B);
  nv.insert(nv.end(), rec_node, rec_node + n_rec);
  SBFWI_CUDA(nodes.alloc(sizeof(int64_t) * nv.size()));
  SBFWI_CUDA(cudaMemcpyAsync(nodes.p, nv.data(), sizeof(int64_t) * nv.size(), cudaMemcpyHostToDevice, st));
  const int64_t ntr = (int64_t)B * n_rec * K;
  double* dtraces = nullptr;
  if (ntr > 0) {
    if (mem == SBFWI_MEM_DEVICE) {
      dtraces = traces;               // written in place
    } else {
      SBFWI_CUDA(traces_owned.alloc(sizeof(double) * ntr));
      dtraces = traces_owned.as<double>();
    }
  }
  RunBuffers rb;
  Stepper f(*md, Mode::Forward, B, K, n_rec, rb, st);
  f.values = values.as<double>(); f.nodes = nodes.as<int64_t>(); f.traces = dtraces;
  int rc = f.init();
  if (rc) return rc;
  std::unique_ptr<sbfwi_fwdstate> fs;
  int64_t c = 0;
  if (keep) {
    fs.reset(new sbfwi_fwdstate());
    fs->model = md; fs->B = B; fs->R = n_rec; fs->K = K;
    fs->rec.assign(rec_node, rec_node + n_rec);
    const int64_t sd = f.state_doubles();
    const int64_t ss = f.store_stride();
    c = ckpt_every;
    if (c == SBFWI_CKPT_AUTO) {
      // memory (K/c) * sd + c * ss * B is least at c = sqrt(K sd / (ss B))
      c = (int64_t)std::ceil(std::sqrt((double)K * (double)sd / ((double)ss * B)));
    }
    c = std::min<int64_t>(c, K);
    if (md->kernel_terms == SBFWI_TERMS_FULL && md->lfe)
      return fail(SBFWI_EUNSUPPORTED, "the comparison method has no radial field for the full kernel's gradient term");
    fs->ckpt_every = c;
    fs->state_doubles = sd;
    fs->tensor_core_path = f.tensor_core_path();
    fs->exact = md->grad_mode == SBFWI_GRAD_EXACT;
    cudaError_t e = cudaSuccess;
    double gb = 0;
    if (c == 0 && fs->exact) {
      // the exact adjoint reads u and u'' of every step (no velocities)
      gb = 2.0 * K * np * B * 8 / 1e9;
      e = store_alloc(fs->store_u, sizeof(double) * (size_t)K * np * B);
      if (e == cudaSuccess) e = fs->store_a.alloc(sizeof(double) * (size_t)K * np * B);
    } else if (c == 0) {
      gb = (double)K * ss * B * 8 / 1e9;
      e = store_alloc(fs->store, sizeof(double) * (size_t)K * ss * B);
      if (e == cudaSuccess && md->kernel_terms == SBFWI_TERMS_FULL) {
        gb *= 2;
        e = fs->store_u.alloc(sizeof(double) * (size_t)K * np * B);
      }
    } else {
      const int64_t nseg = (K + c - 1) / c;
      gb = (double)(nseg - 1) * sd * 8 / 1e9;
      if (nseg > 1) e = store_alloc(fs->store, sizeof(double) * (size_t)(nseg - 1) * sd);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SBFWI_ENOMEM, "not enough device memory to keep the forward state (" + std::to_string(gb) + " GB)");
    }
  }
  if (!keep || c == 0) {
    f.store = (fs && fs->store.p) ? fs->store.as<double>() : nullptr;
    f.store_u = (fs && fs->store_u.p) ? fs->store_u.as<double>() : nullptr;
    f.store_a = (fs && fs->store_a.p) ? fs->store_a.as<double>() : nullptr;
    rc = f.run(0, K);
  } else {
    // checkpoints: the Newmark state before steps c, 2c, ... (before step 0 it is zero)
    const int64_t sd = fs->state_doubles;
    for (int64_t a = 0; a < K && rc == SBFWI_OK; a += c) {
      if (a > 0) rc = f.save_state(fs->store.as<double>() + (a / c - 1) * sd);
      if (rc == SBFWI_OK) rc = f.run(a, std::min(K, a + c));
    }
    fs->values = std::move(values);
    fs->nodes = std::move(nodes);
  }
  if (rc == SBFWI_OK) rc = f.check_status();
  if (rc == SBFWI_OK && ntr > 0 && mem == SBFWI_MEM_HOST) {
    cudaError_t e = cudaMemcpyAsync(traces, dtraces, sizeof(double) * ntr, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy traces");
  }
  if (rc == SBFWI_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "forward solve");
  }
  profiler().resolve();
  if (rc != SBFWI_OK) return rc;
  if (keep) *keep = fs.release();
  return SBFWI_OK;
}

int sbfwi_adjoint_gradient(sbfwi_model* md, sbfwi_fwdstate* fs, const double* residual, int mode, double* grad, int mem,
                           void* stream) {
  if (!md || !fs || !residual || !grad) return fail(SBFWI_EINVAL, "NULL argument");
  if (fs->model != md) return fail(SBFWI_ESTATE, "forward state belongs to another model");
  const bool accumulate = (mode & SBFWI_GRAD_ACCUMULATE) != 0;
  mode &= ~SBFWI_GRAD_ACCUMULATE;
  if (mode != SBFWI_GRAD_KERNEL && mode != SBFWI_GRAD_EXACT) return fail(SBFWI_EINVAL, "unknown gradient mode");
  if (mem != SBFWI_MEM_HOST && mem != SBFWI_MEM_DEVICE) return fail(SBFWI_EINVAL, "unknown mem");
  const bool exact = mode == SBFWI_GRAD_EXACT;
  const int64_t c = fs->ckpt_every;
  if (exact && !fs->exact)
    return fail(SBFWI_ESTATE, "the forward pass was not kept for the exact adjoint: "
                              "call sbfwi_set_gradient_mode(model, SBFWI_GRAD_EXACT) before it");
  if (!exact && c == 0 && !fs->store.p)
    return fail(SBFWI_ESTATE, "the forward pass kept displacements and accelerations for the exact adjoint, "
                              "not the velocities of the paper's kernel");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int B = fs->B, R = fs->R;
  const int64_t K = fs->K, np = md->mesh->n_nodal;
  DevBuf values, nodes;
  const int64_t nres = (int64_t)B * R * K;
  SBFWI_CUDA(values.alloc(sizeof(double) * std::max<int64_t>(nres, 1)));
  if (nres > 0)
    SBFWI_CUDA(cudaMemcpyAsync(values.p, residual, sizeof(double) * nres,
                               mem == SBFWI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  SBFWI_CUDA(nodes.alloc(sizeof(int64_t) * std::max<size_t>(fs->rec.size(), 1)));
  if (R > 0) SBFWI_CUDA(cudaMemcpyAsync(nodes.p, fs->rec.data(), sizeof(int64_t) * R, cudaMemcpyHostToDevice, st));
  RunBuffers rb;
  Stepper adj(*md, exact ? Mode::Exact : Mode::Adjoint, B, K, R, rb, st);
  adj.values = values.as<double>(); adj.nodes = nodes.as<int64_t>();
  int rc = adj.init();
  if (rc) return rc;
  const bool full = !exact && md->kernel_terms == SBFWI_TERMS_FULL;
  if (full && c == 0) {
    if (!fs->store_u.p)
      return fail(SBFWI_ESTATE, "the forward pass kept no displacements: set the full kernel before the forward pass");
    adj.fwd_u = fs->store_u.as<double>();
  }
  if (c == 0) {
    if (exact) {
      adj.fwd_u = fs->store_u.as<double>();
      adj.fwd_a = fs->store_a.as<double>();
      rc = adj.run_exact(0, K);
    } else {
      adj.fwd = fs->store.as<double>();
      rc = adj.run(0, K);
    }
  } else {
    // recompute the forward field one window of c steps at a time from the checkpoints,
    // last window first, and run the adjoint steps that pair with it
    RunBuffers rf;
    Stepper fwd(*md, Mode::Forward, B, K, 0, rf, st);
    fwd.values = fs->values.as<double>(); fwd.nodes = fs->nodes.as<int64_t>();
    rc = fwd.init();
    if (rc) return rc;
    if (fwd.tensor_core_path() != fs->tensor_core_path || fwd.state_doubles() != fs->state_doubles)
      return fail(SBFWI_ESTATE, "the element kernel differs from the one that wrote the checkpoints");
    // the window holds the recomputed velocities (the paper's kernel), plus the displacements
    // for the full kernel's gradient term; the exact adjoint's displacements and accelerations
    DevBuf window, window_a;
    const int64_t ss = (exact || full) ? np : fwd.store_stride();
    cudaError_t e = window.alloc(sizeof(double) * (size_t)c * ss * B);
    if (e == cudaSuccess && (exact || full)) e = window_a.alloc(sizeof(double) * (size_t)c * ss * B);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(SBFWI_ENOMEM, "not enough device memory for one recompute window (" +
                                    std::to_string((exact ? 2.0 : 1.0) * c * ss * B * 8 / 1e9) + " GB)");
    }
    const int64_t nseg = (K + c - 1) / c;
    for (int64_t seg = nseg - 1; seg >= 0 && rc == SBFWI_OK; --seg) {
      const int64_t a = seg * c, b = std::min(K, a + c);
      rc = seg == 0 ? fwd.zero_state() : fwd.restore_state(fs->store.as<double>() + (seg - 1) * fs->state_doubles);
      fwd.store_k0 = a;
      if (exact) {
        fwd.store = nullptr;
        fwd.store_u = window.as<double>();
        fwd.store_a = window_a.as<double>();
      } else {
        fwd.store = window.as<double>();
        if (full) fwd.store_u = window_a.as<double>();
      }
      if (rc == SBFWI_OK) rc = fwd.run(a, b);
      if (exact) {
        adj.fwd_u = window.as<double>(); adj.fwd_a = window_a.as<double>(); adj.fwd_k0 = a;
        if (rc == SBFWI_OK) rc = adj.run_exact(a, b);
      } else {
        adj.fwd = window.as<double>(); adj.fwd_k0 = a;
        if (full) adj.fwd_u = window_a.as<double>();
        if (rc == SBFWI_OK) rc = adj.run(K - b, K - a);
      }
    }
    if (rc == SBFWI_OK) rc = fwd.check_status();
  }
  if (rc == SBFWI_OK && exact) rc = adj.finalize_exact();
  if (rc == SBFWI_OK) rc = adj.check_status();
  if (rc) return rc;
  // the paper's kernel accumulates per shot and applies dt at the end; the exact gradient is
  // already summed over shots (dt is in its misfit adjoint)
  const int Bsum = exact ? 1 : B;
  const double scale = exact ? 1.0 : md->dt;
  DevBuf gn;
  SBFWI_CUDA(gn.alloc(sizeof(double) * np));
  const unsigned blocks = (unsigned)std::min<int64_t>((np + 255) / 256, 152 * 8);
  sum_shots_kernel<<<blocks, 256, 0, st>>>(rb.grad_int.as<double>(), np, Bsum, scale, gn.as<double>(), 0);
  profiler().count(kPhaseOther);
  rc = emit_gradient(*md, gn.as<double>(), grad, mem, accumulate, st);
  profiler().resolve();
  return rc;
}

int sbfwi_misfit(const double* traces, const double* observed, int64_t n, double dt, double* E_out, double* residual_out,
                 int mem, void* stream) {
  if (!traces || !observed || !E_out) return fail(SBFWI_EINVAL, "NULL argument");
  if (n < 0) return fail(SBFWI_EINVAL, "n < 0");
  if (mem != SBFWI_MEM_HOST && mem != SBFWI_MEM_DEVICE) return fail(SBFWI_EINVAL, "unknown mem");
  if (!have_device()) return fail(SBFWI_ECUDA, "no CUDA device");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf dt_, dob, dres, part, eout;
  const double* tr = traces;
  const double* ob = observed;
  double* res = residual_out;
  const int64_t nn = std::max<int64_t>(n, 1);
  if (mem == SBFWI_MEM_HOST) {
    SBFWI_CUDA(dt_.alloc(sizeof(double) * nn));
    SBFWI_CUDA(dob.alloc(sizeof(double) * nn));
    if (n > 0) {
      SBFWI_CUDA(cudaMemcpyAsync(dt_.p, traces, sizeof(double) * n, cudaMemcpyHostToDevice, st));
      SBFWI_CUDA(cudaMemcpyAsync(dob.p, observed, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    }
    tr = dt_.as<double>();
    ob = dob.as<double>();
    if (residual_out) { SBFWI_CUDA(dres.alloc(sizeof(double) * nn)); res = dres.as<double>(); }
  }
  const int parts = 256;
  SBFWI_CUDA(part.alloc(sizeof(double) * parts));
  SBFWI_CUDA(eout.alloc(sizeof(double)));
  misfit_partial_kernel<<<parts, 256, 0, st>>>(tr, ob, n, res, part.as<double>());
  misfit_final_kernel<<<1, 256, 0, st>>>(part.as<double>(), parts, 0.5 * dt, eout.as<double>());
  profiler().count(kPhaseOther, 2);
  SBFWI_CUDA(cudaGetLastError());
  SBFWI_CUDA(cudaMemcpyAsync(E_out, eout.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (mem == SBFWI_MEM_HOST && residual_out && n > 0)
    SBFWI_CUDA(cudaMemcpyAsync(residual_out, res, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  SBFWI_CUDA(cudaStreamSynchronize(st));
  return SBFWI_OK;
}

int sbfwi_selftest_barrier(int32_t n_blocks, int32_t n_absent, int64_t budget_cycles, int32_t rounds, void* stream) {
  if (n_blocks < 1 || n_absent < 0 || n_absent >= n_blocks) return fail(SBFWI_EINVAL, "need 0 <= n_absent < n_blocks");
  if (budget_cycles < 1000 || budget_cycles > 4000000000LL) return fail(SBFWI_EINVAL, "budget_cycles must be in [1e3, 4e9]");
  if (rounds < 1 || rounds > 1000) return fail(SBFWI_EINVAL, "rounds must be in 1..1000");
  if (!have_device()) return fail(SBFWI_ECUDA, "no CUDA device");
  int device = 0, coop = 0, sms = 0, per_sm = 0;
  SBFWI_CUDA(cudaGetDevice(&device));
  SBFWI_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
  SBFWI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  SBFWI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_selftest_kernel, 64, 0));
  if (!coop) return fail(SBFWI_EUNSUPPORTED, "device cannot launch cooperatively");
  if ((int64_t)n_blocks > (int64_t)per_sm * sms) return fail(SBFWI_EINVAL, "n_blocks exceeds the co-resident limit");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevBuf bar, status;
  SBFWI_CUDA(bar.alloc(2 * sizeof(unsigned)));
  SBFWI_CUDA(status.alloc(sizeof(int)));
  SBFWI_CUDA(cudaMemsetAsync(bar.p, 0, bar.bytes, st));
  SBFWI_CUDA(cudaMemsetAsync(status.p, 0, status.bytes, st));
  unsigned* barp = bar.as<unsigned>();
  int* statusp = status.as<int>();
  long long budget = budget_cycles;
  int absent = n_absent, r = rounds;
  void* kargs[] = {&barp, &statusp, &budget, &absent, &r};
  SBFWI_CUDA(cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(n_blocks), dim3(64), kargs, 0, st));
  int code = 0;
  SBFWI_CUDA(cudaMemcpyAsync(&code, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SBFWI_CUDA(cudaStreamSynchronize(st));
  if (code) return fail(SBFWI_ETIMEOUT, "grid barrier self-test: a block did not arrive within the budget");
  return SBFWI_OK;
}


// ---------------------------------------------------------------------------
// sessions (continuous batching)
// ---------------------------------------------------------------------------
int sbfwi_session_create(sbfwi_session** out, sbfwi_model* md, int32_t kind, int32_t slots, int32_t n_rec,
                         const int64_t* rec_node, int32_t window, void* stream) {
  if (!out) return fail(SBFWI_EINVAL, "out is NULL");
  *out = nullptr;
  if (!md) return fail(SBFWI_EINVAL, "model is NULL");
  if (kind != SBFWI_SESSION_FORWARD && kind != SBFWI_SESSION_ADJOINT) return fail(SBFWI_EINVAL, "unknown session kind");
  if (slots < 1 || slots > kMaxShots) return fail(SBFWI_EINVAL, "slots must be in 1..16");
  if (window < 1 || window > 100000) return fail(SBFWI_EINVAL, "window must be in 1..100000");
  if (n_rec < 0 || (n_rec > 0 && !rec_node)) return fail(SBFWI_EINVAL, "receivers need rec_node");
  if (kind == SBFWI_SESSION_ADJOINT && md->kernel_terms == SBFWI_TERMS_FULL)
    return fail(SBFWI_EUNSUPPORTED, "sessions accumulate the velocity kernel only");
  if (md->grad_mode == SBFWI_GRAD_EXACT)
    return fail(SBFWI_EUNSUPPORTED, "sessions run the paper's kernel, not the exact adjoint");
  for (int r = 0; r < n_rec; ++r) {
    if (rec_node[r] < 0 || rec_node[r] >= md->N) return fail(SBFWI_EINVAL, "receiver node out of range");
    for (int r2 = 0; r2 < r; ++r2)
      if (rec_node[r2] == rec_node[r]) return fail(SBFWI_EINVAL, "receiver nodes must be distinct");
  }
  if (!have_device()) return fail(SBFWI_ECUDA, "no CUDA device");
  std::unique_ptr<sbfwi_session> S(new sbfwi_session());
  S->md = md; S->kind = kind; S->B = slots; S->R = n_rec; S->W = window;
  S->st = static_cast<cudaStream_t>(stream);
  S->rec.assign(rec_node, rec_node + n_rec);
  const bool fwd = kind == SBFWI_SESSION_FORWARD;
  S->sp.reset(new Stepper(*md, fwd ? Mode::Forward : Mode::Adjoint, slots, window, n_rec, S->rb, S->st));
  Stepper& sp = *S->sp;
  sp.tasks_own = &S->tasks;
  sp.resume = true;
  // node list: forward B sources (set on admission) then the receivers; adjoint the receivers
  std::vector<int64_t> nv;
  if (fwd) nv.assign(slots, S->rec.empty() ? 0 : S->rec[0]);
  nv.insert(nv.end(), S->rec.begin(), S->rec.end());
  SBFWI_CUDA(S->nodes.alloc(sizeof(int64_t) * std::max<size_t>(nv.size(), 1)));
  if (!nv.empty()) SBFWI_CUDA(cudaMemcpy(S->nodes.p, nv.data(), sizeof(int64_t) * nv.size(), cudaMemcpyHostToDevice));
  int rc = sp.init();
  if (rc) return rc;
  const int64_t nval = fwd ? (int64_t)slots * window : (int64_t)slots * n_rec * window;
  SBFWI_CUDA(S->win_values.alloc(sizeof(double) * std::max<int64_t>(nval, 1)));
  SBFWI_CUDA(cudaMemsetAsync(S->win_values.p, 0, S->win_values.bytes, S->st));
  if (fwd && n_rec > 0) SBFWI_CUDA(S->win_traces.alloc(sizeof(double) * (size_t)slots * n_rec * window));
  if (!fwd) {
    SBFWI_CUDA(S->win_field.alloc(sizeof(double) * (size_t)window * sp.store_stride() * slots));
    sp.fwd = S->win_field.as<double>();
    sp.fwd_k0 = 0;
  }
  sp.values = S->win_values.as<double>();
  sp.nodes = S->nodes.as<int64_t>();
  sp.traces = S->win_traces.as<double>();
  SBFWI_CUDA(S->slots_dev.alloc(sizeof(SlotDev) * slots));
  S->slots.resize(slots);
  S->slots_h.resize(slots);
  if ((rc = S->upload_slots())) return rc;
  *out = S.release();
  return SBFWI_OK;
}

int sbfwi_session_info(const sbfwi_session* S, int64_t* info) {
  if (!S || !info) return fail(SBFWI_EINVAL, "NULL argument");
  info[0] = S->sp->store_stride();
  info[1] = S->kglob;
  info[2] = S->B;
  info[3] = S->W;
  int64_t busy = 0;
  for (const SlotHost& h : S->slots) busy += h.active ? 1 : 0;
  info[4] = busy;
  return SBFWI_OK;
}

void sbfwi_session_destroy(sbfwi_session* S) {
  if (S && S->st) cudaStreamSynchronize(S->st);
  delete S;
}

int sbfwi_session_admit(sbfwi_session* S, int32_t slot, int64_t src_node, const double* values, int64_t K,
                        double* field, int mem) {
  if (!S) return fail(SBFWI_EINVAL, "session is NULL");
  if (slot < 0 || slot >= S->B) return fail(SBFWI_EINVAL, "slot out of range");
  if (S->slots[slot].active) return fail(SBFWI_ESTATE, "slot is busy");
  if (K < 1 || !values) return fail(SBFWI_EINVAL, "need K >= 1 values");
  if (mem != SBFWI_MEM_HOST && mem != SBFWI_MEM_DEVICE) return fail(SBFWI_EINVAL, "unknown mem");
  const bool fwd = S->kind == SBFWI_SESSION_FORWARD;
  if (fwd && (src_node < 0 || src_node >= S->md->N)) return fail(SBFWI_EINVAL, "source node out of range");
  if (!fwd && !field) return fail(SBFWI_EINVAL, "an adjoint slot needs the forward velocities");
  SlotHost& h = S->slots[slot];
  const int64_t nv = fwd ? K : (int64_t)S->R * K;
  SBFWI_CUDA(h.values.alloc(sizeof(double) * std::max<int64_t>(nv, 1)));
  if (nv > 0)
    SBFWI_CUDA(cudaMemcpyAsync(h.values.p, values, sizeof(double) * nv,
                               mem == SBFWI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S->st));
  h.traces.release();
  if (fwd && S->R > 0) {
    SBFWI_CUDA(h.traces.alloc(sizeof(double) * (size_t)S->R * K));
    SBFWI_CUDA(cudaMemsetAsync(h.traces.p, 0, h.traces.bytes, S->st));
  }
  h.field = field;
  h.start = S->kglob; h.K = K; h.active = true; h.finished = false;
  int rc = S->sp->zero_column(slot);
  if (rc) return rc;
  if (fwd) {
    SBFWI_CUDA(cudaMemcpyAsync(S->nodes.as<int64_t>() + slot, &src_node, sizeof(int64_t), cudaMemcpyHostToDevice, S->st));
    if (field && !S->field_used) {
      SBFWI_CUDA(S->win_field.alloc(sizeof(double) * (size_t)S->W * S->sp->store_stride() * S->B));
      S->sp->store = S->win_field.as<double>();
      S->sp->store_k0 = 0;
      S->field_used = true;
    }
  }
  return S->upload_slots();        // synchronises: src_node is read before returning
}

int sbfwi_session_step(sbfwi_session* S, int32_t* finished) {
  if (!S) return fail(SBFWI_EINVAL, "session is NULL");
  const int B = S->B, R = S->R, W = S->W;
  const bool fwd = S->kind == SBFWI_SESSION_FORWARD;
  bool any = false;
  for (const SlotHost& h : S->slots) any = any || (h.active && !h.finished);
  if (any) {
    Profiler& prof = profiler();
    const cudaStream_t st = S->st;
    const SlotDev* sd = S->slots_dev.as<SlotDev>();
    const int64_t nval = fwd ? (int64_t)B * W : (int64_t)B * R * W;
    if (nval > 0) {
      session_sources_kernel<<<(unsigned)std::min<int64_t>((nval + 255) / 256, 152 * 8), 256, 0, st>>>(
          sd, B, R, S->kglob, W, fwd ? 0 : 1, S->win_values.as<double>());
      prof.count(kPhaseOther);
    }
    const int64_t stride = S->sp->store_stride();
    const int64_t nf = (int64_t)W * stride * B;
    if (!fwd) {
      session_field_kernel<<<(unsigned)std::min<int64_t>((nf + 255) / 256, 152 * 16), 256, 0, st>>>(
          sd, B, stride, S->kglob, W, 1, S->win_field.as<double>());
      prof.count(kPhaseOther);
    }
    SBFWI_CUDA(cudaGetLastError());
    int rc = S->sp->run(0, W);
    if (rc == SBFWI_OK) rc = S->sp->check_status();
    if (rc) return rc;
    if (fwd && R > 0) {
      const int64_t nt = (int64_t)B * R * W;
      session_traces_kernel<<<(unsigned)std::min<int64_t>((nt + 255) / 256, 152 * 8), 256, 0, st>>>(
          sd, B, R, S->kglob, W, S->win_traces.as<double>());
      prof.count(kPhaseOther);
    }
    if (fwd && S->field_used) {
      session_field_kernel<<<(unsigned)std::min<int64_t>((nf + 255) / 256, 152 * 16), 256, 0, st>>>(
          sd, B, stride, S->kglob, W, 0, S->win_field.as<double>());
      prof.count(kPhaseOther);
    }
    SBFWI_CUDA(cudaGetLastError());
    SBFWI_CUDA(cudaStreamSynchronize(st));
    profiler().resolve();
    S->kglob += W;
  }
  for (int s = 0; s < B; ++s) {
    SlotHost& h = S->slots[s];
    if (h.active && !h.finished && S->kglob >= h.start + h.K) h.finished = true;
    if (finished) finished[s] = (h.active && h.finished) ? 1 : 0;
  }
  return SBFWI_OK;
}

int sbfwi_session_collect(sbfwi_session* S, int32_t slot, double* out, int mem) {
  if (!S || !out) return fail(SBFWI_EINVAL, "NULL argument");
  if (slot < 0 || slot >= S->B) return fail(SBFWI_EINVAL, "slot out of range");
  if (mem != SBFWI_MEM_HOST && mem != SBFWI_MEM_DEVICE) return fail(SBFWI_EINVAL, "unknown mem");
  SlotHost& h = S->slots[slot];
  if (!h.active || !h.finished) return fail(SBFWI_ESTATE, "slot has no finished request");
  const cudaStream_t st = S->st;
  int rc = SBFWI_OK;
  if (S->kind == SBFWI_SESSION_FORWARD) {
    if (S->R > 0)
      SBFWI_CUDA(cudaMemcpyAsync(out, h.traces.p, sizeof(double) * S->R * h.K,
                                 mem == SBFWI_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    SBFWI_CUDA(cudaStreamSynchronize(st));
  } else {
    Model& md = *S->md;
    const int64_t np = md.mesh->n_nodal;
    DevBuf g;
    SBFWI_CUDA(g.alloc(sizeof(double) * np));
    column_copy_kernel<<<(unsigned)std::min<int64_t>((np + 255) / 256, 152 * 8), 256, 0, st>>>(
        S->rb.grad_int.as<double>(), np, S->B, slot, md.dt, g.as<double>());
    profiler().count(kPhaseOther);
    rc = emit_gradient(md, g.as<double>(), out, mem, false, st);
  }
  h.active = false; h.finished = false;
  h.values.release(); h.traces.release(); h.field = nullptr;
  if (rc == SBFWI_OK) rc = S->upload_slots();
  return rc;
}

}  // extern "C"
