// lhdm_engine.cuh -- device engine of the LHDM / LH nonnegative least-squares
// solver (Algorithms 1-5 of Dessole, Dell'Orto, Marcuzzi).
//
// One solve is one persistent launch.  A "team" of CTAs runs the whole outer
// loop of Algorithm 3: the grid team is every SM of the GPU (one CTA per SM,
// phases separated by a grid barrier with a bounded wait), the CTA team is a
// single CTA that owns one instance of a batch (phases separated by
// __syncthreads).  Every phase spreads its FP64 work over all threads of the
// team; control decisions are recomputed identically by every CTA from data
// published before the last barrier, so all CTAs follow the same path.
//
// Positivity trick (section 3.2, NNLS on [A -A] with x = (x+, x-)): the team
// solves it on the n physical columns.  A passive column carries a sign
// (csign): +1 stands for column j of [A -A], -1 for its twin n + j.  Since
// Q^T(-a) = -Q^T a and a Householder reflector built from -x equals the one
// built from x, R, W, y and x are kept for the physical columns and the signs
// enter only where a sign is tested: the dual value of the pair is |w_j|
// (index j if w_j >= 0, else n + j), y and x of column n + j are -y_j, -x_j.
// The twin of a passive column is not in Z.
//
// State of an instance (section 2.1, whole-matrix variant of section 4.1):
//   W  = Q^T A for the columns in Z (the B and C blocks), m x n, ld ldw;
//        columns in P are not kept current in W - their R column is in R.
//   bt = Q^T b.
//   R  = the nP x nP triangular factor, column of position p stored in slot
//        rslot[p] of a cap x cap array (ld ldr); rows are QR rows.
//   order[p] = column index at position p (QR column order), pos[c] = p or -1.
//   xP[p]    = x at position p.
// The Householder vectors of the current panel live in V (row-major, ld KM).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "lhdm.h"

namespace lhdm {

constexpr int KM = LHDM_KMAX_LIMIT;  // 64
constexpr int NT = 512;              // threads per CTA
constexpr int NW = NT / 32;          // warps per CTA
constexpr int PW = 2112;             // partial-sum slots per CTA (>= KM(KM+1)/2 + 16)
// Slot ranges inside one CTA's partial row.  A range is only rewritten after
// a barrier that follows every read of its previous contents:
//   [0, KM(KM+1)/2)        candidate Gram pairs (DM)
//   [0, 8(KM+1))           panel exchange (dots, second dots, two pivot rows),
//                          double-buffered by exchange parity
//   [P_O1, P_O1 + 8)       outer-loop argmax / maxima / sums
//   P_RS                   residual sum of squares
constexpr int P_O1 = PW - 16;
constexpr int P_RS = PW - 1;
constexpr int TB = 64;               // triangular-solve block
constexpr int SLAB = 16;             // rows per accumulation slab of the pipelined solve
constexpr int INV_PARTS = TB / NW;   // column classes of a diagonal-block inverse (one column per warp)
constexpr int DB = 32;               // downdate block (positions per warp)
constexpr int PACC_COPIES = 4;       // copies of the panel exchange's sums (ranks mod 4)
constexpr int PACC_W = PACC_COPIES * 2 * (KM + 1);  // one exchange buffer (int64 words)
constexpr int NPHASE = 12;
constexpr double EPS = 2.220446049250313e-16;  // 2^-52
constexpr long long WAIT_NS = 4000000000LL;    // default bound on any device-side wait

enum Phase {
  PH_SETUP = 0, PH_DM, PH_PANEL, PH_SOLVE, PH_COMMIT, PH_INNER, PH_RESID, PH_DUAL,
  PH_FEAS, PH_CHAIN, PH_ZROT, PH_ITRSV
};

struct DevParams {
  double tau1, tau2, delta, tol_w;
  int k_max, max_outer;
  int mode;  // LHDM_MODE_*: 0 plain NNLS; 1, 2 the positivity trick on [A -A]
             // (2: with the sign flip of section 4.2 in the inner loop)
};

// Everything a team needs for one instance.  Persistent fields (R, rslot,
// order, xP, r, nP_out) survive the solve for the adjoint.
struct Inst {
  int m, n, lda, cap, ldw, ldr;
  const double* A;
  const double* b;
  double* x_out;
  int* passive_out;
  lhdm_info* info_out;
  // persistent
  double* R;
  int* rslot;
  int* order;
  double* xP;
  double* r;
  int* nP_out;
  // scratch
  double* W;
  double* bt;
  double* yP;
  double* rhs;
  double* w;
  double* u;
  double* anorm;
  double* V;      // >= m x KM, row-major
  double* vtop;   // KM
  double* beta;   // KM
  double* T;      // KM x KM
  double* R22;    // KM x KM
  double* Gm;     // KM x KM
  double* yJ;     // KM
  double* pr;     // KM (panel right-hand side)
  double* part;   // team.size x PW
  long long* pacc;  // 3 x PACC_W: fixed-point sums of the panel exchange
  double* candw;  // team.size x KM
  double* rotc;   // rotation log
  double* rots;
  int* pos;       // n
  int* J;         // KM
  int* candi;     // team.size x KM
  int* candn;     // team.size
  int* ipart;     // team.size x 8
  int* ctl;       // 16 ints of control words
  int* qlist;     // cap: positions removed by the current inner step
  int* csign;     // n: positivity trick, sign of a passive column (+1: column j
                  // of [A -A], -1: its twin n + j); unused otherwise
  double* Dinv;   // ceil(cap/TB) x TB x TB inverses of R's diagonal blocks (null: no pipelined solve)
  double* accb;   // ceil(cap/TB) x TB slab accumulations of the pipelined solve
  int* tflag;     // ceil(cap/TB) block flags, ceil(cap/TB) * TB/SLAB slab flags, ceil(cap/TB) * INV_PARTS inverse flags
  unsigned long long* amask;  // KM acceptance masks
  unsigned* Vd;   // panel reflectors as 7-bit digits: m rows x ND planes x 16 words (bf16 pairs,
                  // 16-byte chunk c of row r at c ^ (r & 7)), null: none
  int* Ver;       // m: row scale exponents of Vd (|V(r, :)| < 2^Ver[r])
  double* phase_ns;           // 2 NPHASE + 1 (may be null): phase times, phase flops,
                              // bf16 MMAs of the tensor-core commit
  int* trace;                 // 6 ints per outer step (may be null)
  int trace_cap;              // rows available in trace
  long long wait_ns;          // bound on a wait for another CTA (ns)
  int bar_extra;              // failure-detection test: arrivals the grid barrier
                              // expects beyond the grid (0 in every normal solve)
  int guard_force;            // test aid: 1 sends every tensor-core commit batch to
                              // FP64 as the accuracy guard would (0 in normal solves)
  DevParams prm;
};

// control words (ctl[])
enum { C_KP = 0, C_DROPS, C_CAND, C_NROT, C_NRUN, C_READY, C_STATUS, C_ERR, C_KK, C_NFLIP,
       C_GUARD1 }; // commit batches the accuracy guard handed to the FP64 path

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Even split of [0, total) into `parts` contiguous ranges.
__device__ __forceinline__ void split(int total, int parts, int idx, int& lo, int& hi) {
  lo = (int)(((long long)total * idx) / parts);
  hi = (int)(((long long)total * (idx + 1)) / parts);
}

// Block-wide sum, same value in every thread, fixed order.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = lane < NW ? sh[lane] : 0.0;
  return warp_sum(t);
}

// (value, index) argmax with lowest index on ties; idx < 0 = empty.
struct ArgMax {
  double v;
  int i;
};
__device__ __forceinline__ ArgMax amax_merge(ArgMax a, ArgMax b) {
  if (b.i < 0) return a;
  if (a.i < 0) return b;
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}
__device__ __forceinline__ ArgMax warp_amax(ArgMax a) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    ArgMax b;
    b.v = __shfl_xor_sync(0xffffffffu, a.v, o);
    b.i = __shfl_xor_sync(0xffffffffu, a.i, o);
    a = amax_merge(a, b);
  }
  return a;
}
__device__ __forceinline__ ArgMax block_amax(ArgMax a, double* shv, int* shi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_amax(a);
  __syncthreads();
  if (lane == 0) { shv[warp] = a.v; shi[warp] = a.i; }
  __syncthreads();
  ArgMax t;
  t.v = lane < NW ? shv[lane] : 0.0;
  t.i = lane < NW ? shi[lane] : -1;
  return warp_amax(t);
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = lane < NW ? sh[lane] : -INFINITY;
  return warp_max(t);
}
__device__ __forceinline__ int block_sum_int(int v, int* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  int t = lane < NW ? sh[lane] : 0;
#pragma unroll
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// ------------------------------------------- FP64 products on bf16 MMA
// A double x with |x| < 2^E is held as the fixed-point integer
// Y = round(|x| 2^(56-E)) < 2^56, cut into ND = 8 digits of 7 bits
// (Y = sum_k d_k 2^(49-7k)), each exactly a bf16 (sign of x).  A product
// of digits is below 2^14, so sums of up to 2^10 of them are exact in the
// FP32 accumulators of the tensor cores.  A dot product is rebuilt from its
// level sums P_lam = sum_{k+l=lam} (digit-pair sums) as
// sum_lam 2^(-7 lam) P_lam over the levels lam <= NLV-1 = 8; the pairs left
// out carry weight below 2^-59 of the operands' scales, so the result is as
// accurate as a dot product in FP64.
constexpr int ND = 8;
constexpr int NLV = ND + 1;

// round(|x| 2^sh) for |x| 2^sh < 2^56 (zero and subnormal x give 0).  Only
// elements at least 2^3 below the scale are rounded, so the result stays
// below 2^56.
__device__ __forceinline__ unsigned long long fix56(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FFu);
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int s = e - 1075 + sh;
  unsigned long long y = 0ull;
  if (s >= 0) y = mant << (s > 3 ? 3 : s);
  else if (s > -64) y = (mant + (1ull << (-s - 1))) >> (-s);
  return e == 0 ? 0ull : y;
}
// exponent bound: |x| < 2^ebound(x); -2000 for zero and subnormals
__device__ __forceinline__ int ebound(double x) {
  const int e = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu);
  return e == 0 ? -2000 : e - 1022;
}
// Y as two 28-bit halves (digits 0-3 in hi, 4-7 in lo)
__device__ __forceinline__ void halves28(unsigned long long y, unsigned& hi, unsigned& lo) {
  hi = (unsigned)(y >> 28);
  lo = (unsigned)y & 0x0FFFFFFFu;
}
// sign words of two values for dig2: (+-1, +-1) and (-+128, -+128) as bf16x2
__device__ __forceinline__ void sign2(bool nega, bool negb, unsigned& sg, unsigned& nb) {
  sg = (nega ? 0xBF80u : 0x3F80u) | ((negb ? 0xBF80u : 0x3F80u) << 16);
  nb = (nega ? 0x4300u : 0xC300u) | ((negb ? 0x4300u : 0xC300u) << 16);
}
// digit at bit offset sh of two half-words as bf16x2 (a low, b high):
// bf16 0x4300 | d is 128 + d, and s (128 + d) - 128 s = s d exactly
__device__ __forceinline__ unsigned dig2(unsigned wa, unsigned wb, int sh, unsigned sg, unsigned nb) {
  const unsigned p = ((wa >> sh) & 0x7Fu) | (((wb >> sh) & 0x7Fu) << 16) | 0x43004300u;
  unsigned r;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(p), "r"(sg), "r"(nb));
  return r;
}
// a bf16 pair times 2^-7 (exact for the 7-bit digits: no bits are lost)
__device__ __forceinline__ unsigned bf16x2_scale_m7(unsigned x) {
  unsigned r;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(0x3C003C00u), "r"(0x80008000u));
  return r;
}
// digit k (0..7) of a value given as 28-bit halves
__device__ __forceinline__ unsigned dig2k(int k, unsigned ha, unsigned la, unsigned hb, unsigned lb, unsigned sg,
                                          unsigned nb) {
  const int sh = 21 - 7 * (k & 3);
  return k < 4 ? dig2(ha, hb, sh, sg, nb) : dig2(la, lb, sh, sg, nb);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void ldsm_x4(unsigned* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(unsigned* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}
// c += a b, m16n8k16, bf16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float* c, const unsigned* a, const unsigned* b) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// 16-byte asynchronous copy global -> shared (zero fill when !ok)
__device__ __forceinline__ void cp16(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(ok ? 16 : 0)
               : "memory");
}
// 8- and 4-byte asynchronous copies global -> shared (zero fill when !ok)
__device__ __forceinline__ void cp8(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(ok ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp4(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// mbarrier and bulk (TMA) copies global -> shared
__device__ __forceinline__ void mbar_init(unsigned long long* mb, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
// bytes and both addresses multiples of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* mb) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mb))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* mb, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 2^e as a double, e in the normal range [-1022, 1023]
__device__ __forceinline__ double pow2n(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
// x 2^e for |e| <= 2044 by one or two exact power-of-two multiplications
// (only a result in the subnormal range is rounded)
__device__ __forceinline__ double scale2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * pow2n(e);
  const int e1 = e / 2;
  return (x * pow2n(e1)) * pow2n(e - e1);
}

// u 2^es, rounded once to nearest (ties to even) like scale2((double)u, es),
// built with integer instructions: on this GPU a conversion to FP64 costs
// one instruction of the FP64 pipe, which the integer pipe does not share.
// Results outside the normal range take the FP64 route.
__device__ __forceinline__ double ll_scaled(long long u, int es) {
  if (u == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)u & 0x8000000000000000ull;
  unsigned long long a = (u < 0) ? 0ull - (unsigned long long)u : (unsigned long long)u;
  const int lz = __clzll(a);
  int e = 63 - lz + es + 1023;  // biased exponent of the leading bit
  if (e < 1 || e > 2045) return scale2((double)u, es);
  a <<= lz;
  unsigned long long m = a >> 11;  // 53 bits, leading bit set
  const unsigned rem = (unsigned)(a & 0x7FFull);
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  if (m >> 53) {  // rounded up to the next power of two
    m >>= 1;
    ++e;
  }
  return __longlong_as_double((long long)(sgn | ((unsigned long long)e << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// Reciprocal and square root for the solver's scalar chains (the panel's
// reflectors, the diagonal reciprocals of the triangular solves, the
// rotation publisher of the downdate).  On this
// GPU one FP64 instruction is 64 cycles of a sub-partition, and the
// correctly rounded division and square root of the compiler take about ten
// each; these take four and five on the dependent path.  The seed is the
// single-precision hardware approximation (rcp.approx / rsqrt.approx, about
// 2^-22) of the mantissa, rebuilt as a double with integer instructions;
// then, for 1/d, two Newton-Raphson steps y += y (1 - d y) (each squares
// the relative error), and for sqrt(s) one Goldschmidt step on (g, h) =
// (s y, y / 2) followed by a Newton correction with the exact remainder
// s - g^2 (Markstein's scheme).  Both end within about one ulp of the
// correctly rounded result (lhdm_debug_fast_math checks this against the
// library's).  Arguments outside the normal range, zero and non-finite ones
// take the library's routines.
__device__ __forceinline__ double rcp_nr(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int E = (int)((b >> 52) & 0x7FFu) - 1023;
  if (E < -1000 || E > 1000) return 1.0 / d;  // also zero, subnormal, inf, nan
  float r;
  const float mf = __uint_as_float(0x3F800000u | (unsigned)((b >> 29) & 0x7FFFFFull));  // |mantissa| in [1, 2)
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(mf));
  const unsigned rb = __float_as_uint(r);
  const long long ye = (long long)(((rb >> 23) & 0xFFu) - 127 - E + 1023);
  double y = __longlong_as_double((long long)(b & 0x8000000000000000ull) | (ye << 52) |
                                  ((long long)(rb & 0x7FFFFFu) << 29));
  double e = fma(-d, y, 1.0);
  y = fma(y, e, y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ double sqrt_gm(double s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(s);
  const int E = (int)((b >> 52) & 0x7FFu) - 1023;
  if (!(s > 0.0) || E < -1000 || E > 1000) return sqrt(s);
  // s = f 2^(2k), f in [1, 4): the seed is rsqrt(f) 2^-k
  const int k = E >> 1;  // floor(E / 2)
  const unsigned fe = (unsigned)(E - 2 * k);  // 0 or 1
  const float mf = __uint_as_float(((127u + fe) << 23) | (unsigned)((b >> 29) & 0x7FFFFFull));
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(mf));
  const unsigned rb = __float_as_uint(r);
  const long long ye = (long long)((rb >> 23) & 0xFFu) - 127 - k + 1023;
  const double y = __longlong_as_double((ye << 52) | ((long long)(rb & 0x7FFFFFu) << 29));
  const double hy = __longlong_as_double(((ye - 1) << 52) | ((long long)(rb & 0x7FFFFFu) << 29));  // y / 2
  double g = s * y;
  const double r1 = fma(-g, hy, 0.5);
  g = fma(g, r1, g);
  const double h = fma(hy, r1, hy);
  const double dr = fma(-g, g, s);
  return fma(dr, h, g);
}

// x with |x| <= 2^(E-1) as a fixed-point integer in units of 2^(E-56)
// (truncated; |q| <= 2^55).  Such integers add exactly and in any order to
// the same sum, and up to 256 of them fit in 64 bits.
__device__ __forceinline__ long long fx_q(double x, int E) { return __double2ll_rz(scale2(x, 56 - E)); }
__device__ __forceinline__ double fx_x(long long q, int E) { return scale2((double)q, E - 56); }

// ---------------------------------------------------------------- teams
// Whole-grid team: one CTA per SM, co-resident (cooperative launch).  The
// barrier counts arrivals on a word that only grows (see arrive_wait); every
// wait is bounded by wait_ns and sets *err on expiry, after which every CTA
// leaves the solve.  `extra` raises the arrival count of the main barrier
// beyond the grid: only the
// failure-detection test sets it, so that no CTA ever releases the barrier and
// every wait runs out.
struct GridTeam {
  int rank, size;
  // [0] arrivals at whole-team barriers, [2] arrivals at sub-team barriers
  // (both zero at launch; [2] is zeroed again after every panel): the k-th
  // barrier completes when its counter reaches the arrivals of barriers
  // 1..k, so an arrival is one release-add and nothing is ever reset
  // inside a barrier
  unsigned int* bar;
  int* err;
  long long wait_ns;
  int extra;  // arrivals a whole-team barrier expects beyond the team
  unsigned int full_target = 0u, sub_target = 0u;
  __device__ __forceinline__ bool sync() {
    full_target += (unsigned)(size + extra);
    return arrive_wait(bar, full_target);
  }
  // barrier of ranks 0 .. n-1 only (the other ranks must not call it)
  __device__ __forceinline__ bool sync_sub(int n) {
    sub_target += (unsigned)n;
    return arrive_wait(bar + 2, sub_target);
  }
  // after a whole-team barrier that follows the last sub-team barrier of a
  // panel (every rank calls it): the sub-team count starts again from zero
  __device__ __forceinline__ void sub_reset() {
    if (rank == 0 && threadIdx.x == 0) atomicExch(bar + 2, 0u);
    sub_target = 0u;
  }
  __device__ __forceinline__ bool arrive_wait(unsigned int* cnt, unsigned int target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      int ok = 1;
      // release: what the CTA wrote before the CTA barrier above is visible
      // to every CTA that acquires a count including this arrival
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt) : "memory");
      const long long t0 = gtimer();
      unsigned int spins = 0;
      for (;;) {
        // err first (relaxed), so that both loads are in flight together
        const int e = *(volatile int*)err;
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
        if (e) { ok = 0; break; }
        if (v >= target) break;
        if ((++spins & 63u) == 0u && gtimer() - t0 > wait_ns) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  }
};

// Single-CTA team (one batch instance per CTA).
struct CtaTeam {
  int rank, size;
  __device__ __forceinline__ bool sync() {
    __threadfence_block();
    __syncthreads();
    return true;
  }
  __device__ __forceinline__ bool sync_sub(int) { return sync(); }
  __device__ __forceinline__ void sub_reset() {}
};

// Flags between CTAs.  A CTA publishes with one thread after a CTA barrier
// (the release covers what every thread wrote before that barrier); a
// waiting thread acquires, and a CTA barrier after the wait passes the
// values on to the other threads.
__device__ __forceinline__ void flag_release(int* flag, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(flag), "r"(v) : "memory");
}
__device__ __forceinline__ int flag_acquire(const int* flag) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
  return v;
}

// Bounded wait until *flag >= target (one thread); false on timeout.
__device__ __forceinline__ bool wait_ge(const int* flag, int target, int* err, long long wait_ns) {
  if (flag_acquire(flag) >= target) return true;
  const long long t0 = gtimer();
  unsigned int spins = 0;
  while (flag_acquire(flag) < target) {
    if ((++spins & 63u) == 0u) {
      if (err && *(volatile int*)err) return false;
      if (gtimer() - t0 > wait_ns) {
        if (err) atomicExch(err, 1);
        return false;
      }
    }
  }
  return true;
}

template <class Team>
struct Engine;

}  // namespace lhdm
