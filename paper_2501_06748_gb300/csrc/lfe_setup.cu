// The comparison method's element matrices on the GPU (Section 3.2, low-frequency
// expansion of the reduced element equation): one CTA per element computes
//   K from the Riccati equation (K - E1) E0^-1 (K - E1^T) - E2 = 0 as Q_q Q_u^-1 for a basis of
//     the bounded solutions of xi d/dxi [u; q] = -Z [u; q], Z = [[E0^-1 E1^T, -E0^-1],
//     [-E2 + E1 E0^-1 E1^T, -E1 E0^-1]]: the stable subspace is the range of
//     (I - sign(Z + I/2)) / 2 (matrix sign function by the determinant-scaled Newton
//     iteration, Roberts' method), its rank must be n_b - 1, a basis by Gram-Schmidt with
//     column pivoting, plus the constant mode [1; 0];
//   M from the Lyapunov equation F M + M G = M0, F = (K - E1) E0^-1 + I,
//     G = E0^-1 (K - E1^T) + I, by the coupled Newton sign iteration (the spectra of F and
//     G are 1 + the bounded modes' exponents, >= 1).
// The same steps as the host routine behind sbfwi_lfe_element_matrices (lfe.cpp), in FP64,
// here for every element of a model in one launch; the model's set-up then assembles
// S_e = K_e + M_e / (beta dt^2) and keeps M_e for the per-step effective sources.
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "prof.h"

namespace sbfwi {
namespace {

struct LfeArgs {
  int nb;                    // stride of the padded per-element matrices
  int64_t e0, E;             // first element of this launch, elements in the model
  const int32_t* nbe;        // [E] n_b of each element
  const double* Emat;        // [E][4][nb][nb] E0, E1, E2, M0
  double a0;                 // 1 / (beta dt^2)
  double* S;                 // [E][nb][nb] out: K + a0 M
  double* Mout;              // [E][nb][nb] out: M
  double* ws;                // workspace, ws_per doubles per element of the launch
  int64_t ws_per;
  int* status;
};

// block-wide maximum of v (every thread passes its value; all threads get the result)
__device__ double block_max(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = red[0];
  for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, red[k]);
  __syncthreads();
  return m;
}

__device__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m += red[k];
  __syncthreads();
  return m;
}

// C (n x m) = A (n x k) B (k x m), row-major, distinct buffers
__device__ void bmm(int n, int k, int m, const double* A, const double* B, double* C) {
  for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
    const int r = t / m, c = t - r * m;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s = fma(A[r * k + l], B[l * m + c], s);
    C[t] = s;
  }
  __syncthreads();
}

// Inv = A^{-1} by Gauss-Jordan with partial pivoting (A destroyed); returns false if a pivot
// vanishes; *logdet = log |det A|
__device__ bool ginv(int n, double* A, double* Inv, double* col, double* red, double* logdet) {
  __shared__ int piv;
  __shared__ double lsum;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) Inv[t] = (t / n == t % n) ? 1.0 : 0.0;
  if (threadIdx.x == 0) lsum = 0.0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int best = k;
      double bv = fabs(A[k * n + k]);
      for (int r = k + 1; r < n; ++r)
        if (fabs(A[r * n + k]) > bv) { bv = fabs(A[r * n + k]); best = r; }
      piv = (bv > 0.0 && isfinite(bv)) ? best : -1;
      if (piv >= 0) lsum += log(bv);
    }
    __syncthreads();
    const int pr = piv;
    if (pr < 0) return false;
    if (pr != k)
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double t1 = A[k * n + c]; A[k * n + c] = A[pr * n + c]; A[pr * n + c] = t1;
        const double t2 = Inv[k * n + c]; Inv[k * n + c] = Inv[pr * n + c]; Inv[pr * n + c] = t2;
      }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) col[r] = A[r * n + k];
    __syncthreads();
    const double pinv = 1.0 / col[k];
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int r = t / n, c = t - r * n;
      if (r == k) continue;
      const double f = col[r] * pinv;
      A[t] = fma(-f, A[k * n + c], A[t]);
      Inv[t] = fma(-f, Inv[k * n + c], Inv[t]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      A[k * n + c] *= pinv;
      Inv[k * n + c] *= pinv;
    }
    __syncthreads();
  }
  if (logdet) *logdet = lsum;
  (void)red;
  return true;
}

__global__ void __launch_bounds__(256) lfe_setup_kernel(LfeArgs a) {
  __shared__ double red[32];
  __shared__ double col[96];
  __shared__ int s_ok, s_best;
  const int64_t e = a.e0 + blockIdx.x;
  if (e >= a.E) return;
  const int nbs = a.nb, n = a.nbe[e], n2 = 2 * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* w = a.ws + (int64_t)blockIdx.x * a.ws_per;
  // workspace: six n2 x n2 matrices, then ten n x n
  double* X = w;
  double* Xi = X + n2 * n2;
  double* T = Xi + n2 * n2;
  double* Pc = T + n2 * n2;            // projector columns, column-major: column c at Pc + c * n2
  double* Qb = Pc + n2 * n2;           // basis vectors, n - 1 of length n2
  double* E0 = Qb + n2 * n2 + n2 * n2;
  double* E1 = E0 + n * n;
  double* E2 = E1 + n * n;
  double* M0 = E2 + n * n;
  double* A = M0 + n * n;              // scratch n x n
  double* Bm = A + n * n;
  double* Cm = Bm + n * n;
  double* Dm = Cm + n * n;
  double* Fm = Dm + n * n;
  double* Gm = Fm + n * n;
  const double* Ee = a.Emat + e * 4 * (int64_t)nbs * nbs;
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, c = t - r * n;
    E0[t] = Ee[r * nbs + c];
    E1[t] = Ee[(int64_t)nbs * nbs + r * nbs + c];
    E2[t] = Ee[2 * (int64_t)nbs * nbs + r * nbs + c];
    M0[t] = Ee[3 * (int64_t)nbs * nbs + r * nbs + c];
  }
  __syncthreads();
  auto fail = [&](int code) {
    if (tid == 0) atomicCAS(a.status, 0, code);
  };
  // E0^-1 (in Dm), E0^-1 E1^T (A), E1 E0^-1 (Bm), E1 E0^-1 E1^T (Cm)
  for (int t = tid; t < n * n; t += nt) T[t] = E0[t];
  __syncthreads();
  if (!ginv(n, T, Dm, col, red, nullptr)) { fail(SBFWI_ESINGULAR); return; }
  for (int t = tid; t < n * n; t += nt) { const int r = t / n, c = t - r * n; Fm[t] = E1[c * n + r]; }   // E1^T
  __syncthreads();
  bmm(n, n, n, Dm, Fm, A);
  bmm(n, n, n, E1, Dm, Bm);
  bmm(n, n, n, Bm, Fm, Cm);
  // X = Z + I/2
  for (int t = tid; t < n2 * n2; t += nt) {
    const int r = t / n2, c = t - r * n2;
    double v;
    if (r < n && c < n) v = A[r * n + c];
    else if (r < n) v = -Dm[r * n + (c - n)];
    else if (c < n) v = -E2[(r - n) * n + c] + Cm[(r - n) * n + c];
    else v = -Bm[(r - n) * n + (c - n)];
    X[t] = v + (r == c ? 0.5 : 0.0);
  }
  __syncthreads();
  // sign(X) by the determinant-scaled Newton iteration
  bool conv = false;
  for (int it = 0; it < 100 && !conv; ++it) {
    for (int t = tid; t < n2 * n2; t += nt) T[t] = X[t];
    __syncthreads();
    double logdet = 0.0;
    if (!ginv(n2, T, Xi, col, red, &logdet)) { fail(SBFWI_ESINGULAR); return; }
    const double cs = it < 8 ? exp(-logdet / n2) : 1.0;
    double diff = 0.0, norm = 0.0;
    for (int t = tid; t < n2 * n2; t += nt) {
      const double nx = 0.5 * (cs * X[t] + Xi[t] / cs);
      diff = fmax(diff, fabs(nx - X[t]));
      norm = fmax(norm, fabs(nx));
      X[t] = nx;
    }
    __syncthreads();
    diff = block_max(diff, red);
    norm = block_max(norm, red);
    conv = diff <= 1e-14 * norm;
  }
  if (!conv) { fail(SBFWI_ESINGULAR); return; }
  // projector P = (I - sign)/2, stored by columns; its trace must be n - 1
  double tr = 0.0;
  for (int t = tid; t < n2 * n2; t += nt) {
    const int r = t / n2, c = t - r * n2;
    const double p = 0.5 * ((r == c ? 1.0 : 0.0) - X[t]);
    Pc[c * n2 + r] = p;
    if (r == c) tr += p;
  }
  __syncthreads();
  tr = block_sum(tr, red);
  if (fabs(tr - (n - 1)) > 0.25) { fail(SBFWI_ESINGULAR); return; }
  // Gram-Schmidt with column pivoting: n - 1 basis vectors, then the remainder must vanish
  // (T holds a "used" flag per column)
  for (int c = tid; c < n2; c += nt) T[c] = 0.0;
  __syncthreads();
  double first = 0.0;
  for (int k = 0; k < n; ++k) {
    // squared norms of the unused columns, one warp per column
    const int wid = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int c = wid; c < n2; c += nw) {
      double s2 = 0.0;
      for (int r = lane; r < n2; r += 32) s2 = fma(Pc[c * n2 + r], Pc[c * n2 + r], s2);
      for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      if (lane == 0) col[c] = T[c] != 0.0 ? -1.0 : s2;
    }
    __syncthreads();
    if (tid == 0) {
      int best = -1;
      double bn = 0.0;
      for (int c = 0; c < n2; ++c)
        if (col[c] > bn) { bn = col[c]; best = c; }
      s_best = best;
      red[0] = bn;
    }
    __syncthreads();
    const int best = s_best;
    const double bn = red[0];
    __syncthreads();
    if (k == n - 1) {
      if (best >= 0 && bn > 1e-16 * first) { fail(SBFWI_ESINGULAR); return; }
      break;
    }
    if (best < 0 || !(bn > 1e-16 * first)) { fail(SBFWI_ESINGULAR); return; }
    if (k == 0) first = bn;
    double* q = Qb + k * n2;
    const double inv = rsqrt(bn);
    for (int r = tid; r < n2; r += nt) q[r] = Pc[best * n2 + r] * inv;
    if (tid == 0) T[best] = 1.0;
    __syncthreads();
    for (int c = wid; c < n2; c += nw) {
      if (T[c] != 0.0) continue;
      double d = 0.0;
      for (int r = lane; r < n2; r += 32) d = fma(q[r], Pc[c * n2 + r], d);
      for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
      for (int r = lane; r < n2; r += 32) Pc[c * n2 + r] = fma(-d, q[r], Pc[c * n2 + r]);
    }
    __syncthreads();
  }
  // K = Q_q Q_u^-1 with the constant mode as the last basis vector
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, k = t - r * n;
    A[t] = k < n - 1 ? Qb[k * n2 + r] : 1.0;          // Q_u
    Bm[t] = k < n - 1 ? Qb[k * n2 + n + r] : 0.0;     // Q_q
  }
  __syncthreads();
  if (!ginv(n, A, Cm, col, red, nullptr)) { fail(SBFWI_ESINGULAR); return; }
  double* Km = A;
  bmm(n, n, n, Bm, Cm, Km);
  // Lyapunov: F = (K - E1) E0^-1 + I, G = E0^-1 (K - E1^T) + I, C = M0
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, c = t - r * n;
    Bm[t] = Km[t] - E1[t];
    Cm[t] = Km[t] - E1[c * n + r];
  }
  __syncthreads();
  bmm(n, n, n, Bm, Dm, Fm);
  bmm(n, n, n, Dm, Cm, Gm);
  for (int k = tid; k < n; k += nt) { Fm[k * n + k] += 1.0; Gm[k * n + k] += 1.0; }
  double* Cl = M0;                                     // C, overwritten in place
  double* Fi = X;                                      // n x n inverses in the big buffers
  double* Gi = Xi;
  double* W1 = Pc;
  double* W2 = Qb;
  __syncthreads();
  conv = false;
  for (int it = 0; it < 100 && !conv; ++it) {
    for (int t = tid; t < n * n; t += nt) { T[t] = Fm[t]; Bm[t] = Gm[t]; }
    __syncthreads();
    double logdet = 0.0;
    if (!ginv(n, T, Fi, col, red, &logdet)) { fail(SBFWI_ESINGULAR); return; }
    if (!ginv(n, Bm, Gi, col, red, nullptr)) { fail(SBFWI_ESINGULAR); return; }
    const double cs = it < 8 ? exp(-logdet / n) : 1.0;
    bmm(n, n, n, Fi, Cl, W1);
    bmm(n, n, n, W1, Gi, W2);
    double diff = 0.0, norm = 0.0;
    for (int t = tid; t < n * n; t += nt) {
      const double nf = 0.5 * (cs * Fm[t] + Fi[t] / cs);
      diff = fmax(diff, fabs(nf - Fm[t]));
      norm = fmax(norm, fabs(nf));
      Fm[t] = nf;
      Gm[t] = 0.5 * (cs * Gm[t] + Gi[t] / cs);
      Cl[t] = 0.5 * (cs * Cl[t] + W2[t] / cs);
    }
    __syncthreads();
    diff = block_max(diff, red);
    norm = block_max(norm, red);
    conv = diff <= 1e-14 * norm;
  }
  if (!conv) { fail(SBFWI_ESINGULAR); return; }
  double* Se = a.S + e * (int64_t)nbs * nbs;
  double* Me = a.Mout + e * (int64_t)nbs * nbs;
  for (int t = tid; t < n * n; t += nt) {
    const int r = t / n, c = t - r * n;
    const double m = 0.5 * Cl[t];
    Me[r * nbs + c] = m;
    Se[r * nbs + c] = fma(a.a0, m, Km[t]);
  }
  (void)s_ok;
}

}  // namespace

// K_e + a0 M_e into S and M_e into M for every element, from the coefficient matrices
// [E][4][nb][nb] (device); S and M zero beyond each element's n_b.  Elements run in chunks
// that bound the workspace.
int lfe_setup_device(Model& md, const double* Emat, double* S, double* M, cudaStream_t st) {
  const Mesh& m = *md.mesh;
  const int nb = m.nb;
  const int64_t E = m.n_elem;
  const int64_t n2 = 2 * (int64_t)nb;
  const int64_t ws_per = 6 * n2 * n2 + 10 * (int64_t)nb * nb + 64;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)((256u << 20) / (ws_per * 8))));
  DevBuf ws, status;
  SBFWI_CUDA(ws.alloc(sizeof(double) * (size_t)ws_per * chunk));
  SBFWI_CUDA(status.alloc(sizeof(int)));
  SBFWI_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st));
  LfeArgs a;
  a.nb = nb; a.E = E; a.nbe = md.dev().nbe.as<int32_t>(); a.Emat = Emat; a.a0 = md.a0;
  a.S = S; a.Mout = M; a.ws = ws.as<double>(); a.ws_per = ws_per; a.status = status.as<int>();
  for (int64_t e0 = 0; e0 < E; e0 += chunk) {
    a.e0 = e0;
    lfe_setup_kernel<<<(unsigned)std::min(chunk, E - e0), 256, 0, st>>>(a);
    profiler().count(kPhaseSetup);
    SBFWI_CUDA(cudaGetLastError());
  }
  int code = 0;
  SBFWI_CUDA(cudaMemcpyAsync(&code, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SBFWI_CUDA(cudaStreamSynchronize(st));
  if (code) return fail(SBFWI_ESINGULAR, "an element's Riccati or Lyapunov solve of the comparison method failed");
  return SBFWI_OK;
}

}  // namespace sbfwi
