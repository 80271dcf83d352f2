// The tensor-core element step for elements padded to 21..32 boundary nodes: the same
// error-free FP16 digit splitting as tc.cu (one warp per element, one mma.sync.m16n8k16
// per digit pair and significance level), with every n_b x n_b operator cut into 2 x 2
// tiles of 16 x 16 and every operand vector into two k-tiles.  A product
// y = A x sums, per row tile, the levels of both k-tiles before one recombination; the
// row exponents span all 32 rows, the column exponent all 32 entries of a shot, so the
// scaling (and the result) is that of one 32 x 32 product.
#include <type_traits>

#include "internal.h"
#include "prof.h"
#include "tc_digits.cuh"

namespace sbfwi {

namespace tc2 {

using namespace tc;
constexpr int kRT = 2;                       // row tiles (and k-tiles)
constexpr int kR = kTile * kRT;              // padded rows
constexpr int kOpFrags = kRT * kRT * kSlices * 32;   // uint4 per operator
constexpr int kWarps = 2;                    // warps (elements) per block

struct WarpSmem {
  uint4 frag[2][2 * kOpFrags];               // two stages of one or two operators
  int exps[2][2 * kR];
  double xch[kR * kCols];
  uint64_t bar[2];                           // the stages' mbarriers
};

__device__ __forceinline__ const uint4* tile(const uint4* op, int rt, int kt) {
  return op + (rt * kRT + kt) * kSlices * 32;
}

// one stage: two bulk copies (fragments, exponents) completing on the stage's mbarrier
__device__ __forceinline__ void stage_ops(WarpSmem& W, int buf, const uint4* src, const int* sexp, int nops, int lane) {
  if (lane == 0) {
    const unsigned fb = (unsigned)(nops * kOpFrags * sizeof(uint4)), eb = (unsigned)(nops * kR * sizeof(int));
    fence_proxy_async();
    mbar_expect_tx(&W.bar[buf], fb + eb);
    bulk_g2s(W.frag[buf], src, fb, &W.bar[buf]);
    bulk_g2s(W.exps[buf], sexp, eb, &W.bar[buf]);
  }
}

}  // namespace tc2

// one warp per operator, as slice_operators_kernel, for 2 x 2 tiles
__global__ void slice_operators2_kernel(SliceArgs a) {
  using namespace tc2;
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
    out = a.frag + w * kOpFrags;
    eout = a.exps + w * kR;
  } else {
    const int64_t k = w - nmat;
    h = a.rt + k * nn;
    out = a.frag_rt + k * kOpFrags;
    eout = a.exps_rt + k * kR;
  }
  auto val = [&](int r, int c) { return (r < nb && c < nb) ? h[(int64_t)r * nb + c] : 0.0; };
  int er = -1100;                                  // lane r owns row r
  for (int c = 0; c < nb; ++c) er = max(er, exp_bound(val(lane, c)));
  const int which = w < nmat ? (int)(w % 3) : 2;
  int shift = 0;
  if (which < 2) {                                 // P, Q: joint row exponents, balancing power a
    const double* hP = which == 0 ? h : h - nn;
    const double* hQ = hP + nn;
    auto vP = [&](int r, int c) { return (r < nb && c < nb) ? hP[(int64_t)r * nb + c] : 0.0; };
    auto vQ = [&](int r, int c) { return (r < nb && c < nb) ? hQ[(int64_t)r * nb + c] : 0.0; };
    int eP = -1100, eQ = -1100;
    for (int c = 0; c < nb; ++c) { eP = max(eP, exp_bound(vP(lane, c))); eQ = max(eQ, exp_bound(vQ(lane, c))); }
    int mP = eP, mQ = eQ;
    for (int off = 16; off > 0; off >>= 1) {
      mP = max(mP, __shfl_xor_sync(0xffffffffu, mP, off));
      mQ = max(mQ, __shfl_xor_sync(0xffffffffu, mQ, off));
    }
    const int bal = (mP > -1100 && mQ > -1100) ? mQ - mP : 0;
    er = max(eP, eQ > -1100 ? eQ - bal : -1100);
    shift = which == 0 ? 0 : bal;
    if (which == 1) eout[lane] = lane == 0 ? bal : 0;
  }
  if (which != 1) eout[lane] = er;
  for (int rt = 0; rt < kRT; ++rt) {
    const int e_lo = __shfl_sync(0xffffffffu, er, rt * kTile + g) + shift;
    const int e_hi = __shfl_sync(0xffffffffu, er, rt * kTile + g + 8) + shift;
    for (int kt = 0; kt < kRT; ++kt) {
      unsigned short dg[8][kSlices];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int hi = (j >> 1) & 1;
        const int r = rt * kTile + g + hi * 8, c = kt * kTile + 2 * t + (j & 1) + (j >> 2) * 8;
        digits(to_fixed(val(r, c), hi ? e_hi : e_lo), dg[j]);
      }
      uint4* o = out + (rt * kRT + kt) * kSlices * 32;
#pragma unroll
      for (int k = 0; k < kSlices; ++k) {
        uint4 v;
        v.x = pack_digits(dg[0][k], dg[1][k]);
        v.y = pack_digits(dg[2][k], dg[3][k]);
        v.z = pack_digits(dg[4][k], dg[5][k]);
        v.w = pack_digits(dg[6][k], dg[7][k]);
        o[k * 32 + lane] = v;
      }
    }
  }
}

// The element step of element_step_tc_kernel with 2 x 2 operator tiles: fused
// back-substitution + Newmark (+ velocity store or gradient) of one step and the forward
// sweep of the next, operator digits of the next radial point prefetched by cp.async.
template <bool kAvgAccel>
__global__ void __launch_bounds__(64, 2) element_step_tc2_kernel(ElemTcArgs a) {
  using namespace tc2;
  extern __shared__ __align__(16) unsigned char tc2_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  WarpSmem& W = reinterpret_cast<WarpSmem*>(tc2_smem)[warp];
  const int64_t idx = (int64_t)blockIdx.x * kWarps + warp;
  if (idx >= a.n_elems) return;
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
  // C-fragment rows of row tile rt: rt*16 + cr[j]; columns cc[j]
  const int cr[4] = {g, g, g + 8, g + 8};
  const int cc[4] = {2 * t, 2 * t + 1, 2 * t, 2 * t + 1};
  bool cok[kRT][4];
  // B-fragment rows of k-tile kt: kt*16 + br[j]; column g
  const int br[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  bool bok[kRT][4];
#pragma unroll
  for (int r = 0; r < kRT; ++r)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cok[r][j] = r * kTile + cr[j] < nb && cc[j] < B;
      bok[r][j] = r * kTile + br[j] < nb && g < B;
    }

  auto c_to_b = [&](const double (&c)[kRT][4], double (&b)[kRT][4]) {
#pragma unroll
    for (int r = 0; r < kRT; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) X[(r * kTile + cr[j]) * kCols + cc[j]] = c[r][j];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kRT; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) b[r][j] = X[(r * kTile + br[j]) * kCols + g];
    __syncwarp();
  };
  auto finish = [&](auto neg, float (&acc)[kRT][kLevels][4], const int* rexp, int f, double (&y)[kRT][4]) {
    const int fc0 = __shfl_sync(0xffffffffu, f, 4 * cc[0]), fc1 = __shfl_sync(0xffffffffu, f, 4 * cc[1]);
#pragma unroll
    for (int r = 0; r < kRT; ++r) {
      const int er0 = rexp[r * kTile + g], er1 = rexp[r * kTile + g + 8];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        y[r][j] = recombine<decltype(neg)::value>(acc[r], j, (j < 2 ? er0 : er1) + ((j & 1) ? fc1 : fc0));
    }
  };
  // y = A x, A's 2 x 2 tiles of digits in shared memory
  auto apply = [&](const uint4* A, const int* rexp, const double (&xb)[kRT][4], double (&y)[kRT][4]) {
    int fl = -1100;
#pragma unroll
    for (int k = 0; k < kRT; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) fl = max(fl, exp_bound(xb[k][j]));
    const int f = column_exponent(fl);
    float acc[kRT][kLevels][4];
#pragma unroll
    for (int r = 0; r < kRT; ++r) zero(acc[r]);
#pragma unroll
    for (int k = 0; k < kRT; ++k) {
      BDigits d;
      split_b(xb[k], f, d);
#pragma unroll
      for (int r = 0; r < kRT; ++r) product(acc[r], tile(A, r, k) + lane, d);
    }
    finish(std::false_type{}, acc, rexp, f, y);
  };
  // -y = -[P | Q 2^-a][v ; q 2^a] (the sweep's q_i directly)
  auto apply_pq = [&](const uint4* Pf, const uint4* Qf, const int* rexp, const int* aexp, const double (&vb)[kRT][4],
                      const double (&qb)[kRT][4], double (&y)[kRT][4]) {
    const int bal = aexp[0];
    int fl = -1100;
#pragma unroll
    for (int k = 0; k < kRT; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) fl = max(fl, max(exp_bound(vb[k][j]), exp_bound(qb[k][j]) + bal));
    const int f = column_exponent(fl);
    float acc[kRT][kLevels][4];
#pragma unroll
    for (int r = 0; r < kRT; ++r) zero(acc[r]);
#pragma unroll
    for (int k = 0; k < kRT; ++k) {
      BDigits d;
      split_b(vb[k], f, d);
#pragma unroll
      for (int r = 0; r < kRT; ++r) product(acc[r], tile(Pf, r, k) + lane, d);
    }
#pragma unroll
    for (int k = 0; k < kRT; ++k) {
      BDigits d;
      split_b(qb[k], f - bal, d);
#pragma unroll
      for (int r = 0; r < kRT; ++r) product(acc[r], tile(Qf, r, k) + lane, d);
    }
    finish(std::true_type{}, acc, rexp, f, y);
  };

  double xb[kRT][4];
  if (a.do_down) {
    const int64_t hop = (int64_t)3 * kOpFrags;
    const uint4* Hsrc = a.frag + ((e * n + (n - 1)) * 3 + 2) * kOpFrags;
    const int* Hexp = a.exps + ((e * n + (n - 1)) * 3 + 2) * kR;
    stage_ops(W, (n - 1) & 1, Hsrc, Hexp, 1, lane);
#pragma unroll
    for (int k = 0; k < kRT; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        xb[k][j] = bok[k][j] ? a.ub[(int64_t)a.dofs[e * nb + k * kTile + br[j]] * B + g] : 0.0;
    for (int i = n - 1; i >= 0; --i) {
      const int buf = i & 1;
      if (i > 0) stage_ops(W, buf ^ 1, Hsrc - (int64_t)(n - i) * hop, Hexp - (int64_t)(n - i) * 3 * kR, 1, lane);
      double qo[kRT][4], zo[kRT][4], vo[kRT][4], fw[kRT][4], gr[kRT][4];
#pragma unroll
      for (int r = 0; r < kRT; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t o = base + (int64_t)i * per + (r * kTile + cr[j]) * B + cc[j];
          qo[r][j] = cok[r][j] ? a.q[o] : 0.0;
          zo[r][j] = cok[r][j] ? a.ud[o] : 0.0;
          vo[r][j] = cok[r][j] ? a.v[o] : 0.0;
          fw[r][j] = (cok[r][j] && a.grad_int) ? a.fwd_int[o] : 0.0;
          gr[r][j] = (cok[r][j] && a.grad_int) ? a.grad_int[o] : 0.0;
        }
      wait_stage(buf);
      double hu[kRT][4];
      apply(W.frag[buf], W.exps[buf], xb, hu);
      double un[kRT][4];
#pragma unroll
      for (int r = 0; r < kRT; ++r)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          un[r][j] = 0.0;
          if (cok[r][j]) {
            const int64_t o = base + (int64_t)i * per + (r * kTile + cr[j]) * B + cc[j];
            const double u_new = qo[r][j] - hu[r][j];
            const double uddn = fma(a.a0, u_new, -vo[r][j]);
            const double udn = fma(a.c2, uddn, zo[r][j]);
            if (kAvgAccel) {                 // z' = z + dt u''_new, v' = v + a1 z' (as tc.cu)
              const double zn = fma(a.dt, uddn, zo[r][j]);
              a.ud[o] = zn;
              a.v[o] = fma(a.a1, zn, vo[r][j]);
            } else {
              a.ud[o] = fma(a.c1, uddn, udn);
              a.v[o] = fma(a.a0, u_new, fma(a.a1, udn, a.a2 * uddn));
            }
            if (a.store_int) a.store_int[o] = udn;
            if (a.grad_int) a.grad_int[o] = fma(fw[r][j], udn, gr[r][j]);   // dt applied at the end
            if (a.u_out) a.u_out[o] = u_new;
            un[r][j] = u_new;
          }
        }
      c_to_b(un, xb);
    }
  }
  if (!a.do_up) return;
  __syncwarp();
  auto stage_up = [&](int i, int buf) {
    if (i < n) stage_ops(W, buf, a.frag + (e * n + i) * 3 * kOpFrags, a.exps + (e * n + i) * 3 * kR, 2, lane);
    else stage_ops(W, buf, a.frag_rt + e * 2 * kOpFrags, a.exps_rt + e * 2 * kR, 2, lane);
  };
  stage_up(0, 0);
  double qb[kRT][4];
#pragma unroll
  for (int k = 0; k < kRT; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) qb[k][j] = 0.0;
  for (int i = 0; i < n; ++i) {
    const int buf = i & 1;
    stage_up(i + 1, buf ^ 1);
    double vb[kRT][4];
#pragma unroll
    for (int k = 0; k < kRT; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        vb[k][j] = bok[k][j] ? a.v[base + (int64_t)i * per + (k * kTile + br[j]) * B + g] : 0.0;
    wait_stage(buf);
    double qc[kRT][4];
    apply_pq(W.frag[buf], W.frag[buf] + kOpFrags, W.exps[buf], W.exps[buf] + kR, vb, qb, qc);
#pragma unroll
    for (int r = 0; r < kRT; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (cok[r][j]) a.q[base + (int64_t)i * per + (r * kTile + cr[j]) * B + cc[j]] = qc[r][j];
        else qc[r][j] = 0.0;
      }
    c_to_b(qc, qb);
  }
  // effective source f_hat = R q_{n-1} + T v_n
  double vb[kRT][4];
#pragma unroll
  for (int k = 0; k < kRT; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      vb[k][j] = 0.0;
      if (bok[k][j]) {
        const int64_t gi = (int64_t)a.dofs[e * nb + k * kTile + br[j]] * B + g;
        vb[k][j] = fma(a.a0, a.ub[gi], fma(a.a1, a.udb[gi], a.a2 * a.uddb[gi]));
      }
    }
  const int bn = n & 1;
  wait_stage(bn);
  double rq[kRT][4], tv[kRT][4];
  apply(W.frag[bn], W.exps[bn], qb, rq);
  apply(W.frag[bn] + kOpFrags, W.exps[bn] + kR, vb, tv);
#pragma unroll
  for (int r = 0; r < kRT; ++r)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (cok[r][j]) a.fhat[(e * nb + r * kTile + cr[j]) * B + cc[j]] = rq[r][j] + tv[r][j];
}

// host side of the two-row-tile variant
int tc2_prepare(Model& md, cudaStream_t st) {
  using namespace tc2;
  const int n = md.n;
  const int64_t E = md.E;
  SBFWI_CUDA(md.tc_frag.alloc(sizeof(uint4) * (size_t)E * n * 3 * kOpFrags));
  SBFWI_CUDA(md.tc_frag_rt.alloc(sizeof(uint4) * (size_t)E * 2 * kOpFrags));
  SBFWI_CUDA(md.tc_exps.alloc(sizeof(int) * (size_t)E * n * 3 * kR));
  SBFWI_CUDA(md.tc_exps_rt.alloc(sizeof(int) * (size_t)E * 2 * kR));
  SliceArgs a;
  a.nb = md.nb; a.n = n; a.E = E;
  a.mats = md.mats.as<double>(); a.rt = md.rt.as<double>();
  a.frag = md.tc_frag.as<uint4>(); a.frag_rt = md.tc_frag_rt.as<uint4>();
  a.exps = md.tc_exps.as<int>(); a.exps_rt = md.tc_exps_rt.as<int>();
  const int64_t warps = E * n * 3 + E * 2;
  slice_operators2_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(a);
  profiler().count(kPhaseSetup);
  SBFWI_CUDA(cudaGetLastError());
  for (const void* f : {(const void*)element_step_tc2_kernel<true>, (const void*)element_step_tc2_kernel<false>})
    SBFWI_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(WarpSmem) * kWarps)));
  md.tc_ready = true;
  md.tc_one_tile = false;
  return SBFWI_OK;
}

int tc2_element_launch(const ElemTcArgs& a, bool avg_accel, cudaStream_t st) {
  using namespace tc2;
  const int smem = (int)(sizeof(WarpSmem) * kWarps);
  const unsigned blocks = (unsigned)((a.n_elems + kWarps - 1) / kWarps);
  if (avg_accel) element_step_tc2_kernel<true><<<blocks, 32 * kWarps, smem, st>>>(a);
  else element_step_tc2_kernel<false><<<blocks, 32 * kWarps, smem, st>>>(a);
  return SBFWI_OK;
}

}  // namespace sbfwi
