// FP64-accurate element operators on the FP16 tensor cores.
//
// GB300 executes FP64 at ~1.2 TFLOP/s but FP16 mma.sync at ~600 TFLOP/s.  The
// per-step element work is three n_b x n_b matrix products with B shots per radial
// point (q_i = -(P_i v_i + Q_i q_{i-1}), u_i = q_i - H_i u_{i+1}, f_hat = R q_{n-1} + T v_n),
// so it runs here as an error-free splitting of the FP64 operands into FP16 digits
// (the splitting idea of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication", Numer. Algorithms 59 (2012)):
//
//  * every row r of a matrix A is scaled by 2^(53 - e_r), |A[r][.]| < 2^e_r, and
//    rounded to an integer of at most 53 bits; every column (shot) of a vector x the
//    same with its own exponent f; P v + Q q is one product of [P | Q 2^-a] and
//    [v ; q 2^a] with a per-point balancing power a (a shared exponent without it
//    loses ~1e-12 relative near the scaling centre, where |P| << |Q|), H u, R q and
//    T v are scaled on their own;
//  * each integer is written in six balanced base-512 digits (|digit| <= 257, exact
//    in FP16): A_int = sum_k a_k 2^(9(6-k)), x_int = sum_l x_l 2^(9(6-l));
//  * the digit products of one significance level L = k + l are summed by
//    mma.sync.m16n8k16 (FP16 in, FP32 accumulate) into one accumulator per level;
//    every partial sum is an integer below 2^24, so the accumulation is exact;
//  * levels L = 2..8 are kept (the dropped ones weigh < 2^-57 of the scale), turned
//    back into integers, summed in int64 with their weights 2^(9(8-L)), the two lowest
//    levels rounded once to the nearest unit, and converted once to FP64:
//    A x ~ 2^(e_r + f - 52) * T'.
//
// The splitting of the vectors and the recombination are integer work; what stays on
// the FP64 pipe is the conversion of each result and the Newmark arithmetic.
// Shapes: n_b <= 16 (padded to the 16 rows/columns of one m16n8k16 tile) and B <= 8
// shots (padded to its 8 columns); one warp per element.  The joint product sums two
// k-tiles into each level: at most 12 digit products of <= 257^2 times 16 terms,
// 1.3e7 < 2^24, still exact in FP32.
#include <cstdint>
#include <cuda_fp16.h>

#include "internal.h"
#include "prof.h"
#include "tc_digits.cuh"

namespace sbfwi {

// ---------------------------------------------------------------------------
// set-up: slices of the per-step operators in mma fragment layout
// ---------------------------------------------------------------------------
// Operators per element and radial point i: P_i, Q_i, H_i (16 x 16 each after
// padding); per element R and T.  Each is stored as kSlices fragments of 32 lanes x
// uint4 with 16 row exponents.
//
// P_i v_i + Q_i q_{i-1} is formed as ONE product [P_i | Q_i 2^-a][v_i ; q_{i-1} 2^a]
// with shared row exponents (over both halves) and a shared column exponent, where the
// balancing power a_i = e(Q_i) - e(P_i) of the two blocks' largest entries brings them
// to the same scale (P ~ 1e-4 and Q ~ 0.5 near the scaling centre, and q ~ |P| v, so
// q 2^a ~ v).  Without the balancing a shared exponent would cost the smaller block a
// dozen bits.  P's exponent slot holds the joint row exponents, Q's slot holds a_i in
// its first entry.  H, R and T are scaled on their own.

__global__ void slice_operators_kernel(SliceArgs a) {
  using namespace tc;
  // one warp per operator: warps 0..E*n*3-1 are (e, i, P|Q|H), then E*2 warps of (e, R|T)
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int nb = a.nb, n = a.n;
  const int64_t nn = (int64_t)nb * nb;
  const int64_t nmat = a.E * n * 3;
  if (w >= nmat + a.E * 2) return;
  const double* h;
  uint4* out;
  int* eout;
  if (w < nmat) {
    h = a.mats + w * nn;
    out = a.frag + w * kSlices * 32;
    eout = a.exps + w * 16;
  } else {
    const int64_t k = w - nmat;
    h = a.rt + k * nn;
    out = a.frag_rt + k * kSlices * 32;
    eout = a.exps_rt + k * 16;
  }
  auto val = [&](int r, int c) { return (r < nb && c < nb) ? h[(int64_t)r * nb + c] : 0.0; };
  int er = -1100;           // lanes 0..15 own one row each
  if (lane < 16)
    for (int c = 0; c < nb; ++c) er = max(er, exp_bound(val(lane, c)));
  // P or Q of a radial point: joint row exponents with the balancing power a
  const int which = w < nmat ? (int)(w % 3) : 2;
  int shift = 0;            // this operator's digits are taken at row exponent + shift
  if (which < 2) {
    const double* hP = which == 0 ? h : h - nn;
    const double* hQ = hP + nn;
    auto vP = [&](int r, int c) { return (r < nb && c < nb) ? hP[(int64_t)r * nb + c] : 0.0; };
    auto vQ = [&](int r, int c) { return (r < nb && c < nb) ? hQ[(int64_t)r * nb + c] : 0.0; };
    int eP = -1100, eQ = -1100;
    if (lane < 16)
      for (int c = 0; c < nb; ++c) { eP = max(eP, exp_bound(vP(lane, c))); eQ = max(eQ, exp_bound(vQ(lane, c))); }
    int mP = eP, mQ = eQ;
    for (int off = 16; off > 0; off >>= 1) {
      mP = max(mP, __shfl_xor_sync(0xffffffffu, mP, off));
      mQ = max(mQ, __shfl_xor_sync(0xffffffffu, mQ, off));
    }
    const int bal = (mP > -1100 && mQ > -1100) ? mQ - mP : 0;
    er = max(eP, eQ > -1100 ? eQ - bal : -1100);
    shift = which == 0 ? 0 : bal;
    if (which == 1 && lane == 0) eout[0] = bal;
    if (which == 1 && lane > 0 && lane < 16) eout[lane] = 0;
  }
  if (lane < 16 && which != 1) eout[lane] = er;
  const int e_lo = __shfl_sync(0xffffffffu, er, g) + shift, e_hi = __shfl_sync(0xffffffffu, er, g + 8) + shift;
  // fragment entries: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1), then columns + 8
  unsigned short dg[8][kSlices];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int r = g + ((j >> 1) & 1) * 8, c = 2 * t + (j & 1) + (j >> 2) * 8;
    digits(to_fixed(val(r, c), r < 8 ? e_lo : e_hi), dg[j]);
  }
#pragma unroll
  for (int k = 0; k < kSlices; ++k) {
    uint4 v;
    v.x = pack_digits(dg[0][k], dg[1][k]);
    v.y = pack_digits(dg[2][k], dg[3][k]);
    v.z = pack_digits(dg[4][k], dg[5][k]);
    v.w = pack_digits(dg[6][k], dg[7][k]);
    out[k * 32 + lane] = v;
  }
}

// ---------------------------------------------------------------------------
// element step on the tensor cores (one warp per element)
// ---------------------------------------------------------------------------

namespace tc {

// One pipeline stage: the digit fragments of one or two operators and their row
// exponents, brought in by two bulk copies (fragments, exponents) that complete on the
// stage's mbarrier; lane 0 issues them.
constexpr int kStageFrags = 2 * kSlices * 32;     // uint4
struct WarpSmem {
  uint4 frag[2][kStageFrags];
  int exps[2][32];
  double xch[kTile * kCols];
  uint64_t bar[2];
};
constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ void stage_ops(WarpSmem& W, int buf, const uint4* src, const int* sexp, int nops,
                                          int lane) {
  if (lane == 0) {
    const unsigned fb = (unsigned)(nops * kSlices * 32 * sizeof(uint4)), eb = (unsigned)(nops * 16 * sizeof(int));
    fence_proxy_async();                  // the warp's earlier reads of this stage come first
    mbar_expect_tx(&W.bar[buf], fb + eb);
    bulk_g2s(W.frag[buf], src, fb, &W.bar[buf]);
    bulk_g2s(W.exps[buf], sexp, eb, &W.bar[buf]);
  }
}

}  // namespace tc

// One warp per element.  The operator digits of the next radial point are copied to
// shared memory (bulk copies on mbarriers, two stages) while the current point computes,
// and each point's state is loaded before its products, so the memory latency overlaps
// the tensor-core and integer work instead of stalling every radial point.
template <bool kAvgAccel>
__global__ void __launch_bounds__(128, 4) element_step_tc_kernel(ElemTcArgs a) {
  using namespace tc;
  extern __shared__ __align__(16) unsigned char tc_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  WarpSmem& W = reinterpret_cast<WarpSmem*>(tc_smem)[warp];
  const int64_t idx = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (idx >= a.n_elems) return;               // whole warp leaves together
  const int64_t e = a.elems ? (int64_t)a.elems[idx] : idx;
  if (lane == 0) {
    mbar_init(&W.bar[0], 1);
    mbar_init(&W.bar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();
  unsigned phase = 0;                         // bit b: parity of stage b's next completion
  auto wait_stage = [&](int b) {
    mbar_wait(&W.bar[b], (phase >> b) & 1u, a.status);
    phase ^= 1u << b;
  };
  const int nb = a.nb, n = a.n, B = a.B;
  const int per = nb * B;
  double* X = W.xch;
  const int64_t base = e * (int64_t)n * per;
  // C-fragment positions of this lane: (row, col) = (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
  const int cr[4] = {g, g, g + 8, g + 8};
  const int cc[4] = {2 * t, 2 * t + 1, 2 * t, 2 * t + 1};
  bool cok[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) cok[j] = cr[j] < nb && cc[j] < B;
  // B-fragment positions: (row, col) = (2t, g), (2t+1, g), (2t+8, g), (2t+9, g)
  const int br[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  bool bok[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) bok[j] = br[j] < nb && g < B;

  // C layout -> B layout through the warp's shared tile
  auto c_to_b = [&](const double (&c)[4], double (&b)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) X[cr[j] * kCols + cc[j]] = c[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = X[br[j] * kCols + g];
    __syncwarp();
  };
  auto col_exp_b = [&](const double (&b)[4]) {
    int f = -1100;
#pragma unroll
    for (int j = 0; j < 4; ++j) f = max(f, exp_bound(b[j]));
    return column_exponent(f);
  };
  // one product y = A x with A's row exponents (rows g, g+8) and x's column exponent,
  // A's digits in shared memory; returned in C layout
  auto apply = [&](const uint4* A, const int* rexp, const double (&xbv)[4], double (&y)[4]) {
    const int f = col_exp_b(xbv);
    BDigits d;
    split_b(xbv, f, d);
    float acc[kLevels][4];
    zero(acc);
    product(acc, A + lane, d);
    const int er0 = rexp[g], er1 = rexp[g + 8];
    const int fc0 = __shfl_sync(0xffffffffu, f, 4 * cc[0]), fc1 = __shfl_sync(0xffffffffu, f, 4 * cc[1]);
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = recombine(acc, j, (j < 2 ? er0 : er1) + ((j & 1) ? fc1 : fc0));
  };

  // -y = -[P | Q 2^-a][v ; q 2^a] for one radial point (the sweep's q_i directly): P's
  // and Q's digits in shared memory, joint row exponents in rexp, a in aexp[0]; returned
  // in C layout
  auto apply_pq = [&](const uint4* Pf, const uint4* Qf, const int* rexp, const int* aexp, const double (&vbv)[4],
                      const double (&qbv)[4], double (&y)[4]) {
    const int bal = aexp[0];
    int fl = -1100;
#pragma unroll
    for (int j = 0; j < 4; ++j) fl = max(fl, max(exp_bound(vbv[j]), exp_bound(qbv[j]) + bal));
    const int f = column_exponent(fl);
    BDigits dv, dq;
    split_b(vbv, f, dv);
    split_b(qbv, f - bal, dq);
    float acc[kLevels][4];
    zero(acc);
    product(acc, Pf + lane, dv);
    product(acc, Qf + lane, dq);
    const int er0 = rexp[g], er1 = rexp[g + 8];
    const int fc0 = __shfl_sync(0xffffffffu, f, 4 * cc[0]), fc1 = __shfl_sync(0xffffffffu, f, 4 * cc[1]);
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = recombine<true>(acc, j, (j < 2 ? er0 : er1) + ((j & 1) ? fc1 : fc0));
  };

  double xb[4];       // the operand of the next product, B layout
  if (a.do_down) {
    const int64_t hop = (int64_t)3 * kSlices * 32;       // uint4 between radial points
    const uint4* Hsrc = a.frag + ((e * n + (n - 1)) * 3 + 2) * kSlices * 32;
    const int* Hexp = a.exps + ((e * n + (n - 1)) * 3 + 2) * 16;
    stage_ops(W, (n - 1) & 1, Hsrc, Hexp, 1, lane);
#pragma unroll
    for (int j = 0; j < 4; ++j) xb[j] = bok[j] ? a.ub[(int64_t)a.dofs[e * nb + br[j]] * B + g] : 0.0;
    for (int i = n - 1; i >= 0; --i) {
      const int buf = i & 1;
      if (i > 0) stage_ops(W, buf ^ 1, Hsrc - (int64_t)(n - i) * hop, Hexp - (int64_t)(n - i) * 48, 1, lane);
      // the state of this radial point, loaded ahead of the product
      double zo[4], vo[4], qo[4], fw[4], gr[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t o = base + (int64_t)i * per + cr[j] * B + cc[j];
        zo[j] = cok[j] ? a.ud[o] : 0.0;
        vo[j] = cok[j] ? a.v[o] : 0.0;
        qo[j] = cok[j] ? a.q[o] : 0.0;
        fw[j] = (cok[j] && a.grad_int) ? a.fwd_int[o] : 0.0;
        gr[j] = (cok[j] && a.grad_int) ? a.grad_int[o] : 0.0;
      }
      wait_stage(buf);
      double hu[4];
      apply(W.frag[buf], W.exps[buf], xb, hu);
      double un[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        un[j] = 0.0;
        if (cok[j]) {
          const int64_t o = base + (int64_t)i * per + cr[j] * B + cc[j];
          const double u_new = qo[j] - hu[j];
          const double uddn = fma(a.a0, u_new, -vo[j]);
          const double udn = fma(a.c2, uddn, zo[j]);
          // the interior displacement is not kept: the predictor v carries it
          // the interior u', u'' are not kept either: the Newmark update needs only
          // z = u' + dt (1 - gamma) u'' of the old state, the same value the update
          // would form from u' and u'' (same rounding)
          // average acceleration (beta = 1/4, gamma = 1/2): z' = z + dt u''_new and the new
          // predictor a0 u_new + a1 u'_new + u''_new equals v + a1 z' (one FMA instead of two)
          if (kAvgAccel) {
            const double zn = fma(a.dt, uddn, zo[j]);
            a.ud[o] = zn;
            a.v[o] = fma(a.a1, zn, vo[j]);
          } else {
            a.ud[o] = fma(a.c1, uddn, udn);
            a.v[o] = fma(a.a0, u_new, fma(a.a1, udn, a.a2 * uddn));
          }
          if (a.store_int) a.store_int[o] = udn;
          if (a.grad_int) a.grad_int[o] = fma(fw[j], udn, gr[j]);    // dt applied at the end
          if (a.u_out) a.u_out[o] = u_new;
          un[j] = u_new;
        }
      }
      c_to_b(un, xb);     // ends with __syncwarp: the stage just read may be refilled
    }
  }
  if (!a.do_up) return;
  __syncwarp();
  // forward sweep: q_i = -(P_i v_i + Q_i q_{i-1}); stage i holds P_i and Q_i, stage n R and T
  auto stage_up = [&](int i, int buf) {
    if (i < n) stage_ops(W, buf, a.frag + (e * n + i) * 3 * kSlices * 32, a.exps + (e * n + i) * 3 * 16, 2, lane);
    else stage_ops(W, buf, a.frag_rt + e * 2 * kSlices * 32, a.exps_rt + e * 32, 2, lane);
  };
  stage_up(0, 0);
  double vnext[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) vnext[j] = bok[j] ? a.v[base + br[j] * B + g] : 0.0;
  double qb[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i) {
    const int buf = i & 1;
    stage_up(i + 1, buf ^ 1);
    double vb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      vb[j] = vnext[j];
      vnext[j] = (i + 1 < n && bok[j]) ? a.v[base + (int64_t)(i + 1) * per + br[j] * B + g] : 0.0;
    }
    wait_stage(buf);
    double qc[4];
    apply_pq(W.frag[buf], W.frag[buf] + kSlices * 32, W.exps[buf], W.exps[buf] + 16, vb, qb, qc);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (cok[j]) a.q[base + (int64_t)i * per + cr[j] * B + cc[j]] = qc[j];
      else qc[j] = 0.0;
    }
    c_to_b(qc, qb);
  }
  // effective source: f_hat = R q_{n-1} + T v_n, v_n the predictor of the boundary state
  double vb[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    vb[j] = 0.0;
    if (bok[j]) {
      const int64_t gi = (int64_t)a.dofs[e * nb + br[j]] * B + g;
      vb[j] = fma(a.a0, a.ub[gi], fma(a.a1, a.udb[gi], a.a2 * a.uddb[gi]));
    }
  }
  const int bn = n & 1;
  wait_stage(bn);
  double rq[4], tv[4];
  apply(W.frag[bn], W.exps[bn], qb, rq);
  apply(W.frag[bn] + kSlices * 32, W.exps[bn] + 16, vb, tv);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (cok[j]) a.fhat[(e * nb + cr[j]) * B + cc[j]] = rq[j] + tv[j];
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
// Padded n_b 17..20 stays on the FP64 kernel: two 16-row tiles then do 4x the digit work
// of one for at most 1.6x the entries, and on the batching meshes the FP64 kernel was
// faster at n_b = 18 (6.6 s against 8.0 s per step of the p = 3 mesh) while the two-tile
// kernel was faster at n_b = 30 (12.5 s against 21.9 s of the p = 5 mesh).
bool tc_supported(int nb, int B) {
  return (nb <= tc::kTile || (nb >= kTwoTileMinNb && nb <= 2 * tc::kTile)) && B <= tc::kCols;
}
bool tc_available(int nb, int B) { return nb <= 2 * tc::kTile && B <= tc::kCols; }

int tc_prepare(Model& md, cudaStream_t st) {
  using namespace tc;
  if (md.nb > kTile) return tc2_prepare(md, st);
  return tc_prepare_one_tile(md, st);
}

// One-tile digits of every element's operators (their top-left 16 x 16 block; for a mesh
// padded beyond 16 this is the whole operator of its elements with n_b <= 16, whose padded
// rows and columns are zero)
int tc_prepare_one_tile(Model& md, cudaStream_t st) {
  using namespace tc;
  const int nb = md.nb, n = md.n;
  const int64_t E = md.E;
  SBFWI_CUDA(md.tc_frag.alloc(sizeof(uint4) * (size_t)E * n * 3 * kSlices * 32));
  SBFWI_CUDA(md.tc_frag_rt.alloc(sizeof(uint4) * (size_t)E * 2 * kSlices * 32));
  SBFWI_CUDA(md.tc_exps.alloc(sizeof(int) * (size_t)E * n * 3 * 16));
  SBFWI_CUDA(md.tc_exps_rt.alloc(sizeof(int) * (size_t)E * 2 * 16));
  SliceArgs a;
  a.nb = nb; a.n = n; a.E = E;
  a.mats = md.mats.as<double>(); a.rt = md.rt.as<double>();
  a.frag = md.tc_frag.as<uint4>(); a.frag_rt = md.tc_frag_rt.as<uint4>();
  a.exps = md.tc_exps.as<int>(); a.exps_rt = md.tc_exps_rt.as<int>();
  const int64_t warps = E * n * 3 + E * 2;
  slice_operators_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(a);
  profiler().count(kPhaseSetup);
  SBFWI_CUDA(cudaGetLastError());
  // the element kernel's two-stage operator pipeline needs more than the default 48 KiB
  for (const void* f : {(const void*)element_step_tc_kernel<true>, (const void*)element_step_tc_kernel<false>})
    SBFWI_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(WarpSmem) * kWarpsPerBlock)));
  md.tc_ready = true;
  md.tc_one_tile = nb > kTile;
  return SBFWI_OK;
}

int tc_element_launch(const Model& md, int B, int down, int up, double* u, double* ud, double* udd, double* v,
                      const double* ub, const double* udb, const double* uddb, double* q, double* fhat,
                      double* store_int, const double* fwd_int, double* grad_int, double* u_out, cudaStream_t st,
                      const int32_t* elems, int64_t n_elems, int* status) {
  ElemTcArgs a;
  a.nb = md.nb; a.n = md.n; a.B = B; a.E = md.E;
  a.a0 = md.a0; a.a1 = md.a1; a.a2 = md.a2; a.c1 = md.c1; a.c2 = md.c2; a.dt = md.dt;
  a.frag = md.tc_frag.as<uint4>(); a.frag_rt = md.tc_frag_rt.as<uint4>();
  a.exps = md.tc_exps.as<int>(); a.exps_rt = md.tc_exps_rt.as<int>();
  a.dofs = md.dev().dofs.as<int32_t>();
  a.u = u; a.ud = ud; a.udd = udd; a.v = v; a.ub = ub; a.udb = udb; a.uddb = uddb; a.q = q; a.fhat = fhat;
  a.do_down = down; a.do_up = up;
  a.store_int = store_int; a.fwd_int = fwd_int; a.grad_int = grad_int; a.u_out = u_out;
  a.elems = elems; a.n_elems = elems ? n_elems : md.E;
  a.status = status;
  if (a.n_elems == 0) return SBFWI_OK;
  // one 16-row tile: n_b <= 16, or the elements of n_b <= 16 of a mesh padded beyond (the
  // one-tile digits of its operators, prepared by tc_prepare_one_tile)
  if (md.nb > tc::kTile && !md.tc_one_tile) return tc2_element_launch(a, md.a2 == 1.0 && md.c1 == md.c2, st);
  const int smem = (int)(sizeof(tc::WarpSmem) * tc::kWarpsPerBlock);   // attribute set by tc_prepare
  const unsigned blocks = (unsigned)((a.n_elems + tc::kWarpsPerBlock - 1) / tc::kWarpsPerBlock);
  // average acceleration (beta = 1/4, gamma = 1/2): the shorter predictor update
  if (md.a2 == 1.0 && md.c1 == md.c2) element_step_tc_kernel<true><<<blocks, 32 * tc::kWarpsPerBlock, smem, st>>>(a);
  else element_step_tc_kernel<false><<<blocks, 32 * tc::kWarpsPerBlock, smem, st>>>(a);
  return SBFWI_OK;
}

}  // namespace sbfwi
