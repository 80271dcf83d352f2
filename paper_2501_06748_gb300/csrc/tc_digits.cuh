// FP16 digit splitting of FP64 operands for the tensor-core element kernels (shared by
// the one- and two-row-tile kernels): binary64 fields to fixed point, balanced base-512
// digits, m16n8k16 products per significance level, exact integer recombination, and
// the cp.async helpers of the operator pipeline.  The method is described in tc.cu.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>

#include "internal.h"

namespace sbfwi {

namespace tc {

constexpr int kSlices = 6;      // base-512 digits per operand
constexpr int kLevels = 7;      // significance levels kept: k + l = 2..8
constexpr int kTile = 16;       // rows / inner dimension of one mma tile
constexpr int kCols = 8;        // shots of one mma tile

// round(a * 2^(53 - e)) for |a| < 2^e, from the binary64 fields (integer work only)
__device__ __forceinline__ long long to_fixed(double a, int e) {
  const long long bits = __double_as_longlong(a);
  if ((bits & 0x7FFFFFFFFFFFFFFFLL) == 0) return 0;
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long mant = bits & 0x000FFFFFFFFFFFFFLL;
  int ex_eff = ex;
  if (ex == 0) ex_eff = 1;              // subnormal
  else mant |= 0x0010000000000000LL;
  // right shift of the 53-bit significand; |a| < 2^e makes it >= 0
  const int sh = e + 1022 - ex_eff;
  long long v;
  if (sh <= 0) v = mant;
  else if (sh >= 60) v = 0;
  else v = (mant + (1LL << (sh - 1))) >> sh;
  return bits < 0 ? -v : v;
}

// exponent e with |a| < 2^e (for a != 0); very small for a == 0 (integer work only)
__device__ __forceinline__ int exp_bound(double a) {
  const long long bits = __double_as_longlong(a);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return (bits & 0x7FFFFFFFFFFFFFFFLL) == 0 ? -1100 : -1021;
  return ex - 1022;
}

// t * 2^E for results outside the normal range (never met by the path's fields): kept
// out of line so that its FP64 conversion is not evaluated speculatively on the hot path
static __device__ __noinline__ double int_to_double_scaled_slow(long long t, int E) { return ldexp((double)t, E); }

// t * 2^E as a binary64, rounded to nearest-even like a conversion of t, built with
// integer operations (the scaling by 2^E is exact unless the result is subnormal)
__device__ __forceinline__ double int_to_double_scaled(long long t, int E) {
  if (t == 0) return 0.0;
  const unsigned long long sign = t < 0 ? 0x8000000000000000ULL : 0ULL;
  unsigned long long m = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
  const int lz = __clzll((long long)m);
  m <<= lz;                                   // top bit at position 63
  unsigned long long hi = m >> 11;            // 53 bits
  const unsigned long long rem = m & 0x7FFULL;
  if (rem > 0x400ULL || (rem == 0x400ULL && (hi & 1ULL))) ++hi;
  int bexp = E - lz + 11 + 52 + 1023;
  if (hi == (1ULL << 53)) { hi >>= 1; ++bexp; }
  if (bexp >= 1 && bexp <= 2046)
    return __longlong_as_double((long long)(sign | ((unsigned long long)bexp << 52) | (hi & 0x000FFFFFFFFFFFFFULL)));
  return int_to_double_scaled_slow(t, E);
}

// six balanced base-512 digits, most significant first, as FP16 bit patterns of 1536 + d
// The 54-bit recurrence runs on two 32-bit halves: the low 27 bits give the three
// least significant digits and a carry (0 or 1) into the high half, which gives the
// rest -- the same digits as the recurrence on the whole integer.
__device__ __forceinline__ void digits(long long v, unsigned short (&h)[kSlices]) {
  int lo = (int)(v & ((1LL << 27) - 1));      // 0 .. 2^27 - 1
  int hi = (int)(v >> 27);                    // |hi| < 2^26 (arithmetic shift)
#pragma unroll
  for (int k = kSlices - 1; k >= kSlices - 3; --k) {
    const int d = ((lo + 256) & 511) - 256;
    lo = (lo - d) >> 9;
    h[k] = (unsigned short)(0x6600 + d);
  }
  hi += lo;                                   // carry of the low half
#pragma unroll
  for (int k = kSlices - 4; k >= 1; --k) {
    const int d = ((hi + 256) & 511) - 256;
    hi = (hi - d) >> 9;
    h[k] = (unsigned short)(0x6600 + d);
  }
  h[0] = (unsigned short)(0x6600 + hi);
}

// two FP16 patterns of 1536 + d packed in a register -> the pair (d0, d1) as half2
__device__ __forceinline__ unsigned pack_digits(unsigned short lo, unsigned short hi) {
  const unsigned u = (unsigned)lo | ((unsigned)hi << 16);
  __half2 h = *reinterpret_cast<const __half2*>(&u);
  h = __hsub2(h, __halves2half2(__ushort_as_half(0x6600), __ushort_as_half(0x6600)));
  return *reinterpret_cast<const unsigned*>(&h);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint4& a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// Sum of the levels as an int64 with weight 2^-52 relative to 2^(e_r + f).  Levels
// 2..6 are added exactly; levels 7 and 8 are summed exactly apart and rounded once to
// the nearest unit (flooring them with shifts biases every product by about -1 unit,
// which the energy-conserving time loop then accumulates).
// (kNeg: the negated sum, negated in the integer domain -- rounding is symmetric, so the
// result is bit for bit the negation of the kNeg = false one.)
template <bool kNeg = false>
__device__ __forceinline__ double recombine(const float (&acc)[kLevels][4], int j, int e) {
  long long t = 0;
  t += (long long)__float2int_rn(acc[0][j]) << 36;
  t += (long long)__float2int_rn(acc[1][j]) << 27;
  t += (long long)__float2int_rn(acc[2][j]) << 18;
  t += (long long)__float2int_rn(acc[3][j]) << 9;
  t += (long long)__float2int_rn(acc[4][j]);
  const long long low = ((long long)__float2int_rn(acc[5][j]) << 9) + (long long)__float2int_rn(acc[6][j]);
  t += (low + (1LL << 17)) >> 18;
  return int_to_double_scaled(kNeg ? -t : t, e - 52);
}

// Digits of an operand held in the B-fragment layout of m16n8k16: lane (g, t) holds
// rows 2t, 2t+1, 2t+8, 2t+9 of column g.  f is that column's exponent.
struct BDigits {
  unsigned r[kSlices][2];
};

__device__ __forceinline__ void split_b(const double (&x)[4], int f, BDigits& d) {
  unsigned short h[4][kSlices];
#pragma unroll
  for (int j = 0; j < 4; ++j) digits(to_fixed(x[j], f), h[j]);
#pragma unroll
  for (int k = 0; k < kSlices; ++k) {
    d.r[k][0] = pack_digits(h[0][k], h[1][k]);
    d.r[k][1] = pack_digits(h[2][k], h[3][k]);
  }
}

// column exponent: max over the four lanes of a column group (lanes 4g..4g+3)
__device__ __forceinline__ int column_exponent(int e) {
  e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
  e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
  return e;
}

// acc[L] += sum_{k + l = L} A_k x_l over the kept levels; A slices in fragment layout
__device__ __forceinline__ void product(float (&acc)[kLevels][4], const uint4* Aslices, const BDigits& x) {
#pragma unroll
  for (int k = 0; k < kSlices; ++k) {
    const uint4 a = Aslices[k * 32];
#pragma unroll
    for (int l = 0; l < kSlices; ++l)
      if (k + l < kLevels) mma16816(acc[k + l], a, x.r[l][0], x.r[l][1]);
  }
}

__device__ __forceinline__ void zero(float (&acc)[kLevels][4]) {
#pragma unroll
  for (int L = 0; L < kLevels; ++L)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[L][j] = 0.f;
}


// Bulk global -> shared copies by the TMA engine (cp.async.bulk), completing on an mbarrier
// in shared memory: one thread arms the barrier with the byte count and issues the copies;
// every consumer waits on the barrier's phase.  Addresses and sizes are multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// the barrier initialisation visible to the TMA engine before its first use
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// shared memory that the warp read through ordinary loads may now be overwritten by the TMA engine
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n}\n"
               ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_addr(smem)), "l"(gmem), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// wait until the barrier has completed the phase with this parity; bounded: after about
// 2^24 polls (tens of ms) it records SBFWI_ETIMEOUT in *status and gives up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* status) {
  const unsigned a = smem_addr(bar);
  for (int it = 0; it < (1 << 24); ++it) {
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
  }
  if (status) atomicCAS(status, 0, -4 /* SBFWI_ETIMEOUT */);
  return false;
}

}  // namespace tc

// kernel arguments of the operator slicing and the element step (both tile shapes)
struct SliceArgs {
  int nb, n;
  int64_t E;
  const double* mats;     // [E][n][3][nb][nb]
  const double* rt;       // [E][2][nb][nb]
  uint4* frag;            // [E][n][3: P, Q, H][tiles][kSlices][32], tiles = 1 (n_b <= 16) or 4 (<= 32)
  uint4* frag_rt;         // [E][2: R, T][tiles][kSlices][32]
  int* exps;              // [E][n][3][16 or 32] row exponents
  int* exps_rt;           // [E][2][16 or 32]
};

struct ElemTcArgs {
  int nb, n, B;
  int64_t E;
  double a0, a1, a2, c1, c2, dt;
  const uint4* frag;
  const uint4* frag_rt;
  const int* exps;
  const int* exps_rt;
  const int32_t* dofs;
  double* u; double* ud; double* udd; double* v;          // interior state [E][n][nb][B]: this kernel
                                                          // keeps v (predictor) in v and z = u' + dt (1 - gamma) u''
                                                          // in ud; u and udd are unused
  const double* ub; const double* udb; const double* uddb;
  double* q;
  double* fhat;
  int do_down, do_up;
  double* store_int;
  const double* fwd_int;
  double* grad_int;
  double* u_out;          // full Frechet kernel: the new interior displacements (store or adjoint field)
  // the elements this launch steps: elems[0..n_elems) (an element class of a mesh with
  // uneven elements), or all E elements when elems is NULL
  const int32_t* elems;
  int64_t n_elems;
  int* status;            // a bounded wait that gives up records SBFWI_ETIMEOUT here (nullable)
};

// elements padded to 21..32 boundary nodes (tc2.cu)
constexpr int kTwoTileMinNb = 21;
int tc2_prepare(Model& md, cudaStream_t st);
int tc2_element_launch(const ElemTcArgs& a, bool avg_accel, cudaStream_t st);

}  // namespace sbfwi
