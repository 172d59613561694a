// lhdm_solve.cuh -- the outer loop of Algorithm 3 (LHDM) / Algorithm 1 (LH)
// as team-generic device code.  See lhdm_engine.cuh for the state layout.
#pragma once

#include "lhdm_engine.cuh"

namespace lhdm {

// Dynamic shared memory per CTA (bytes) used by the phases below.
constexpr int DYN_SMEM = 160 * 1024;
constexpr int CAND_LOCAL_MAX = 2048;     // local DM candidates per CTA
constexpr int CAND_STAGE = 4096;         // merged candidates staged per pass
constexpr int ROT_STAGE = 2048;          // rotations staged per pass

// Orderable key of a positive double (dual values of DM candidates are > 0).
__device__ __forceinline__ unsigned long long wkey(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
// a better than b: larger w, then smaller index.
__device__ __forceinline__ bool better(unsigned long long ka, int ia, unsigned long long kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

template <class Team>
struct Engine {
  Team& tm;
  const Inst& I;
  double* dyn;
  int tid, lane, warp;

  // uniform control state (identical in every thread of every CTA)
  int nP = 0, n_outer = 0, n_inner = 0, n_drop = 0, rank_limited = 0, status = LHDM_OK;
  double tol_w = 0.0;
  int jsel = -1, n_elig = 0, kk = 0, kp = 0;
  double wmax = 0.0, umax = 0.0, wz_any = -INFINITY, rsq = 0.0;
  double amax = 0.0, bsq = 0.0;
  int nonfinite = 0;
  bool failed = false;
  bool vd_ok = false;  // the current panel's reflector digits are in Vd/Ver
  int kdm = 0, removed = 0, inner_step = 0;
  int inv_valid = 0;  // positions whose diagonal-block inverse column is current
  int tepoch = 0;     // pipelined-solve calls in this launch (flag values)
  int sgn = 0;        // I.prm.mode: 0 plain NNLS, 1 positivity trick, 2 with sign flip
  int nx = 0;         // columns of the problem solved: n, or 2n for [A -A]
  int n_flip = 0;     // sign flips (mode 2)

  // phase timing (rank 0, thread 0)
  long long t_last = 0;
  int cur_phase = -1;
  // per-phase device time and algorithmic FP64 flops (rank 0, thread 0),
  // in shared memory so that no per-thread array forces the engine's state
  // into local memory
  double* phf;

  __device__ Engine(Team& t, const Inst& inst, double* d) : tm(t), I(inst), dyn(d) {
    tid = threadIdx.x;
    lane = tid & 31;
    warp = tid >> 5;
    sgn = I.prm.mode;
    nx = sgn ? 2 * I.n : I.n;
    __shared__ double s_phf[2 * NPHASE];
    phf = s_phf;
    if (tid == 0)
      for (int i = 0; i < 2 * NPHASE; ++i) s_phf[i] = 0.0;
  }

  // Counts algorithmic flops (an FMA is 2) of a phase; uniform state only.
  __device__ __forceinline__ void flops(int p, double f) {
    if (I.phase_ns && tm.rank == 0 && tid == 0) phf[NPHASE + p] += f;
  }

  __device__ __forceinline__ void phase(int p) {
    if (I.phase_ns && tm.rank == 0 && tid == 0) {
      const long long t = gtimer();
      if (cur_phase >= 0) phf[cur_phase] += (double)(t - t_last);
      t_last = t;
      cur_phase = p;
    }
  }

  __device__ __forceinline__ bool sync() {
    if (failed) return false;
    if (!tm.sync()) {
      failed = true;
      status = LHDM_ERR_TIMEOUT;
      return false;
    }
    return true;
  }

  // Positivity trick: the index in [A -A] of physical column c when its dual
  // value is w, the physical column of an index, and the sign of position p.
  __device__ __forceinline__ int ext_of(int c, double w) const { return (sgn && w < 0.0) ? c + I.n : c; }
  __device__ __forceinline__ int phys(int e) const { return e >= I.n ? e - I.n : e; }
  __device__ __forceinline__ double pos_sign(int p) const {
    return sgn ? (double)ldcg(I.csign + ldcg(I.order + p)) : 1.0;
  }

  __device__ __forceinline__ double* Rcol(int slot) const { return I.R + (size_t)slot * I.ldr; }
  __device__ __forceinline__ double* Wcol(int c) const { return I.W + (size_t)c * I.ldw; }

  // Flags of the pipelined solve start at zero in every launch (a barrier
  // must follow before the first solve).
  // A slab sum of the pipelined triangular solve not yet written: a NaN
  // payload no arithmetic produces (results carry the canonical quiet NaN).
  static constexpr long long ACC_EMPTY = 0x7ff4dead0000beefLL;
  __device__ void clear_tri_flags() {
    if (!I.tflag) return;
    const int nbk = (I.cap + TB - 1) / TB, nfl = nbk * (1 + TB / SLAB + INV_PARTS);
    for (int i = tm.rank * NT + tid; i < nfl; i += tm.size * NT) I.tflag[i] = 0;
    for (int i = tm.rank * NT + tid; i < nbk * TB; i += tm.size * NT) I.accb[i] = __longlong_as_double(ACC_EMPTY);
  }

  // ------------------------------------------------------------ setup
  // Algorithm 3, first lines: x = 0, w = A^T b, u = column norms of A; W = A.
  __device__ void setup() {
    __shared__ double sh[32];
    __shared__ int shi[32];
    const int m = I.m, n = I.n;
    int c0, c1;
    split(n, tm.size, tm.rank, c0, c1);
    int bad = 0;
    double am = 0.0;
    for (int c = c0 + warp; c < c1; c += NW) {
      const double* a = I.A + (size_t)c * I.lda;
      double* wc = Wcol(c);
      double s2 = 0.0, sb = 0.0;
      for (int i = lane; i < m; i += 32) {
        const double v = __ldg(a + i);
        wc[i] = v;
        bad |= !isfinite(v);
        s2 = fma(v, v, s2);
        sb = fma(v, __ldg(I.b + i), sb);
      }
      s2 = warp_sum(s2);
      sb = warp_sum(sb);
      const double an = sqrt(s2);
      am = fmax(am, an);
      if (lane == 0) {
        I.anorm[c] = an;
        I.u[c] = an;
        I.w[c] = sb;
        I.pos[c] = -1;
      }
    }
    int r0, r1;
    split(m, tm.size, tm.rank, r0, r1);
    double bs = 0.0;
    for (int i = r0 + tid; i < r1; i += NT) {
      const double v = __ldg(I.b + i);
      bad |= !isfinite(v);
      I.bt[i] = v;
      I.r[i] = v;
      bs = fma(v, v, bs);
    }
    int p0, p1;
    split(I.cap, tm.size, tm.rank, p0, p1);
    for (int p = p0 + tid; p < p1; p += NT) {
      I.xP[p] = 0.0;
      I.yP[p] = 0.0;
      I.rslot[p] = p;
      I.order[p] = -1;
    }
    if (tm.rank == 0 && tid < 16) I.ctl[tid] = 0;
    if (tm.rank == 0)
      for (int e = tid; e < PACC_W; e += NT) I.pacc[e] = 0;  // the panel exchange's first sums
    if (tm.rank == 0 && tid == 0 && I.phase_ns) I.phase_ns[2 * NPHASE] = 0.0;  // MMA count
    clear_tri_flags();
    am = block_max(am, sh);
    bs = block_sum(bs, sh);
    bad = block_sum_int(bad, shi);
    // O1 partial of the first outer step (u = ||a_j||, everything in Z)
    o1_partial(am, bs, (double)bad);
  }

  // Per-CTA partial of the outer-loop test and of the DM maxima over the
  // CTA's column range: argmax of w over the eligible part of Z (lowest
  // index on ties), max u over it, max w over all of Z, eligible count.
  // Slots 5..7 carry extra sums (amax / ||r||^2 / non-finite count).
  // The CTA's columns are its range of [0, n), or the given list of Z
  // columns (the ones it just computed w and u for).  Warp 0 alone scans
  // them (a handful per CTA) and folds the maxima with shuffles: FP64
  // reductions on every warp would cost more than the scan.
  __device__ void o1_partial(double s5, double s6, double s7, const int* list = nullptr, int nlist = 0) {
    __syncthreads();
    if (warp == 0) {
      int c0, c1;
      if (list) {
        c0 = 0;
        c1 = nlist;
      } else {
        split(I.n, tm.size, tm.rank, c0, c1);
      }
      ArgMax best{0.0, -1};
      double um = -INFINITY, wz = -INFINITY;
      int ne = 0;
      for (int k = c0 + lane; k < c1; k += 32) {
        const int c = list ? list[k] : k;
        const int pc = ldcg(I.pos + c);
        const double wc = ldcg(I.w + c), uc = ldcg(I.u + c), an = ldcg(I.anorm + c);
        if (pc >= 0) continue;
        const double wa = sgn ? fabs(wc) : wc;  // the better twin's dual value
        wz = fmax(wz, wa);
        if (uc > (100.0 * EPS) * an) {
          ++ne;
          best = amax_merge(best, ArgMax{wa, ext_of(c, wc)});
          um = fmax(um, uc);
        }
      }
      best = warp_amax(best);
      um = warp_max(um);
      wz = warp_max(wz);
#pragma unroll
      for (int o = 16; o; o >>= 1) ne += __shfl_xor_sync(0xffffffffu, ne, o);
      if (lane == 0) {
        double* p = I.part + (size_t)tm.rank * PW + P_O1;
        p[0] = best.v;
        p[1] = (double)best.i;
        p[2] = um;
        p[3] = wz;
        p[4] = (double)ne;
        p[5] = s5;
        p[6] = s6;
        p[7] = s7;
      }
    }
  }

  // Combines the O1 partials of every CTA (same order everywhere): warp f
  // folds field f of the team (all of a lane's loads in flight at once),
  // warp 0 the argmax pair.
  __device__ double o1_fold(int f, bool is_max) {
    double acc = is_max ? -INFINITY : 0.0;
    for (int t0 = 0; t0 < tm.size; t0 += 32 * 8) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int t = t0 + lane + 32 * j;
        v[j] = (t < tm.size) ? ldcg(I.part + (size_t)t * PW + P_O1 + f) : (is_max ? -INFINITY : 0.0);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) acc = is_max ? fmax(acc, v[j]) : acc + v[j];
    }
    return is_max ? warp_max(acc) : warp_sum(acc);
  }

  __device__ void o1_reduce(bool first) {
    __shared__ double s_d[8];
    __shared__ int s_i[2];
    if (warp == 0) {
      ArgMax best{0.0, -1};
      for (int t0 = 0; t0 < tm.size; t0 += 32 * 8) {
        double v[8], ix[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int t = t0 + lane + 32 * j;
          v[j] = (t < tm.size) ? ldcg(I.part + (size_t)t * PW + P_O1) : 0.0;
          ix[j] = (t < tm.size) ? ldcg(I.part + (size_t)t * PW + P_O1 + 1) : -1.0;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) best = amax_merge(best, ArgMax{v[j], (int)ix[j]});
      }
      best = warp_amax(best);
      if (lane == 0) {
        s_d[0] = best.v;
        s_i[0] = best.i;
      }
    } else if (warp <= 6) {
      // warp 1: max u, 2: max w over Z, 3: eligible count, 4: slot 5 (max on
      // the first call, else sum), 5: slot 6 (sum), 6: slot 7 (sum)
      const int f = warp + 1;
      const bool is_max = (f == 2 || f == 3 || (f == 5 && first));
      const double r = o1_fold(f, is_max);
      if (lane == 0) {
        if (f == 4) s_i[1] = (int)r;
        else s_d[f == 2 ? 1 : f == 3 ? 2 : f - 2] = r;
      }
    }
    __syncthreads();
    wmax = s_d[0];
    umax = s_d[1];
    wz_any = s_d[2];
    jsel = s_i[0];
    n_elig = s_i[1];
    if (first) {
      amax = s_d[3];
      bsq = s_d[4];
      rsq = bsq;
      nonfinite = (int)s_d[5];
    } else {
      rsq = s_d[4];
    }
    __syncthreads();
  }

  // ------------------------------------------------------------ DM
  // Algorithm 2 on C = W[nP:m, Z]: candidates above both thresholds, the
  // first k_max-1 by w (descending; index ascending), cosines of the
  // projected columns, greedy |theta| < delta.  Leaves J in s_J, |J| in kk.
  __device__ bool dm_select(int* s_J) {
    const int km = I.prm.k_max;
    const int kc_max = km - 1;
    const int jp = phys(jsel);
    if (tid == 0) s_J[0] = jp;
    kk = 1;
    if (km <= 1) {
      __syncthreads();
      return true;
    }
    const double thr_w = I.prm.tau1 * wmax;
    const double thr_u = I.prm.tau2 * umax;
    // (a) local candidates of this CTA's column range, locally ranked
    {
      unsigned long long* s_k = reinterpret_cast<unsigned long long*>(dyn);
      int* s_c = reinterpret_cast<int*>(s_k + CAND_LOCAL_MAX);
      __shared__ int s_cnt;
      if (tid == 0) s_cnt = 0;
      __syncthreads();
      int c0, c1;
      split(I.n, tm.size, tm.rank, c0, c1);
      for (int c = c0 + tid; c < c1; c += NT) {
        if (c == jp || ldcg(I.pos + c) >= 0) continue;
        const double wc = ldcg(I.w + c), uc = ldcg(I.u + c), an = ldcg(I.anorm + c);
        const double wa = sgn ? fabs(wc) : wc;
        if (uc > (100.0 * EPS) * an && wa >= thr_w && uc >= thr_u) {
          const int k = atomicAdd(&s_cnt, 1);
          if (k < CAND_LOCAL_MAX) {
            s_k[k] = wkey(wa);
            s_c[k] = ext_of(c, wc);  // ties go to the lower index of [A -A]
          }
        }
      }
      __syncthreads();
      const int cnt = min(s_cnt, CAND_LOCAL_MAX);
      for (int k = tid; k < cnt; k += NT) {
        const unsigned long long kk0 = s_k[k];
        const int ck = s_c[k];
        int rk = 0;
        for (int q = 0; q < cnt; ++q) rk += better(s_k[q], s_c[q], kk0, ck);
        if (rk < kc_max) {
          I.candw[(size_t)tm.rank * KM + rk] = __longlong_as_double((long long)kk0);
          I.candi[(size_t)tm.rank * KM + rk] = ck;
        }
      }
      if (tid == 0) I.candn[tm.rank] = min(cnt, kc_max);
    }
    if (!sync()) return false;
    // (b) merge the sorted local lists: global rank by counting better ones
    __shared__ int s_off[1024 + 1];
    __shared__ int s_kc;
    {
      // prefix offsets of the per-CTA lists (team size <= 1024): the counts
      // are loaded at once (one L2 round trip), then a warp-wide scan
      if (warp == 0) {
        int run = 0;
        for (int j0 = 0; j0 * 32 < tm.size; j0 += 8) {
          int cntv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int t = (j0 + j) * 32 + lane;
            cntv[j] = (t < tm.size) ? ldcg(I.candn + t) : 0;
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            int inc = cntv[j];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int y = __shfl_up_sync(0xffffffffu, inc, o);
              if (lane >= o) inc += y;
            }
            const int t = (j0 + j) * 32 + lane;
            if (t < tm.size) s_off[t] = run + inc - cntv[j];
            run += __shfl_sync(0xffffffffu, inc, 31);
          }
        }
        if (lane == 0) {
          s_off[tm.size] = run;
          s_kc = min(run, kc_max);
        }
      }
      __syncthreads();
      const int total = s_off[tm.size];
      int e0, e1;
      split(total, tm.size, tm.rank, e0, e1);
      unsigned long long* s_k = reinterpret_cast<unsigned long long*>(dyn);
      int* s_c = reinterpret_cast<int*>(s_k + CAND_STAGE);
      // the list and position of merged candidate g (binary search of the
      // offsets)
      auto locate = [&](int g, int& t, int& q) {
        int lo = 0, hi = tm.size;  // s_off[lo] <= g < s_off[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_off[mid] <= g) lo = mid;
          else hi = mid;
        }
        t = lo;
        q = g - s_off[lo];
      };
      // my elements (about total / size): a group of 16 threads per element
      // counts the better candidates, each thread a 16th of them, over the
      // staged passes; the counts are added in the group at the end
      const int mine = e1 - e0;
      const int grp = tid >> 4, sub = tid & 15;
      for (int eb = 0; eb < mine; eb += NT / 16) {
        const int me = eb + grp;
        unsigned long long my_key = 0;
        int my_c = -1;
        if (me < mine) {
          int t, q;
          locate(e0 + me, t, q);
          my_key = wkey(ldcg(I.candw + (size_t)t * KM + q));
          my_c = ldcg(I.candi + (size_t)t * KM + q);
        }
        int cnt = 0;
        for (int base = 0; base < total; base += CAND_STAGE) {
          const int nst = min(CAND_STAGE, total - base);
          __syncthreads();
          for (int k = tid; k < nst; k += NT) {
            int t, q;
            locate(base + k, t, q);
            s_k[k] = wkey(ldcg(I.candw + (size_t)t * KM + q));
            s_c[k] = ldcg(I.candi + (size_t)t * KM + q);
          }
          __syncthreads();
          if (me < mine)
            for (int k = sub; k < nst; k += 16) cnt += better(s_k[k], s_c[k], my_key, my_c);
        }
#pragma unroll
        for (int o = 8; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (me < mine && sub == 0 && cnt < kc_max) I.J[1 + cnt] = my_c;
      }
      if (tm.rank == 0 && tid == 0) I.J[0] = jsel;
    }
    if (!sync()) return false;
    const int kc = s_kc;
    const int KK = kc + 1;
    if (tid < KK) s_J[tid] = phys(ldcg(I.J + tid));
    __syncthreads();
    if (KK == 1) return true;
    // (c) partial Gram matrix of the projected candidates over this CTA's rows
    const int L = I.m - nP;
    const int npair = KK * (KK + 1) / 2;
    flops(PH_DM, 2.0 * npair * (double)L);
    {
      int q0, q1;
      split(L, tm.size, tm.rank, q0, q1);
      double* s_C = dyn;  // 32 x KK
      double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      int pa[5], pb[5];
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        const int p = tid + s * NT;
        pa[s] = -1;
        pb[s] = -1;
        if (p < npair) {
          // pair p -> (a, b), a <= b, row-major upper triangle
          int a = 0, rem = p;
          while (rem >= KK - a) { rem -= KK - a; ++a; }
          pa[s] = a;
          pb[s] = a + rem;
        }
      }
      for (int rb = q0; rb < q1; rb += 32) {
        const int nr = min(32, q1 - rb);
        __syncthreads();
        for (int e = tid; e < nr * KK; e += NT) {
          const int rr = e / KK, a = e - rr * KK;
          s_C[rr * KK + a] = ldcg(Wcol(s_J[a]) + nP + rb + rr);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          if (pa[s] < 0) continue;
          double t = acc[s];
          for (int rr = 0; rr < nr; ++rr) t = fma(s_C[rr * KK + pa[s]], s_C[rr * KK + pb[s]], t);
          acc[s] = t;
        }
      }
#pragma unroll
      for (int s = 0; s < 5; ++s)
        if (pa[s] >= 0) I.part[(size_t)tm.rank * PW + tid + s * NT] = acc[s];
    }
    if (!sync()) return false;
    // (d) reduce the pairs (one warp per pair, lanes over CTAs)
    {
      const int gw = tm.rank * NW + warp, nwt = tm.size * NW;
      for (int p = gw; p < npair; p += nwt) {
        double s = 0.0;
        for (int t = lane; t < tm.size; t += 32) s += ldcg(I.part + (size_t)t * PW + p);
        s = warp_sum(s);
        if (lane == 0) {
          int a = 0, rem = p;
          while (rem >= KK - a) { rem -= KK - a; ++a; }
          const int bb = a + rem;
          I.Gm[a * KM + bb] = s;
          I.Gm[bb * KM + a] = s;
        }
      }
    }
    if (!sync()) return false;
    // (e) cosine test and greedy selection (every CTA, identical)
    {
      __shared__ double s_d[KM];
      __shared__ unsigned long long s_mask[KM];
      if (tid < KK) {
        s_d[tid] = sqrt_gm(ldcg(I.Gm + tid * KM + tid));
        s_mask[tid] = 0ull;
      }
      __syncthreads();
      // |theta_al| = |G_al| / (d_a d_l) < delta, tested without the division
      // (d > 0: every candidate is eligible, u_j > 100 eps ||a_j||)
      for (int p = tid; p < KK * KK; p += NT) {
        const int a = p / KK, l = p - a * KK;
        if (l >= a) continue;
        if (fabs(ldcg(I.Gm + a * KM + l)) < I.prm.delta * (s_d[a] * s_d[l])) atomicOr(&s_mask[a], 1ull << l);
      }
      __syncthreads();
      __shared__ int s_sel[KM];
      __shared__ int s_nsel;
      if (tid == 0) {
        unsigned long long jm = 1ull;
        int ns = 1;
        s_sel[0] = 0;
        for (int a = 1; a < KK; ++a)
          if ((s_mask[a] & jm) == jm) {
            jm |= 1ull << a;
            s_sel[ns++] = a;
          }
        s_nsel = ns;
      }
      __syncthreads();
      const int ns = s_nsel;
      int pick = -1;
      if (tid < ns) pick = s_J[s_sel[tid]];
      __syncthreads();
      if (tid < ns) s_J[tid] = pick;
      kk = ns;
      __syncthreads();
    }
    return true;
  }

  // ------------------------------------------------------------ panel
  // Algorithm 4 on the trailing rows of the chosen columns: one Householder
  // reflector per column in J order (house() as in the oracle), with T of
  // the compact WY form accumulated alongside.  Rows are split over CTAs;
  // each reflector costs one team barrier.
  __device__ bool panel(const int* s_J) {
    vd_ok = false;
    const int L = I.m - nP;
    if (kk > L) kk = L;
    int q0, q1;
    split(L, tm.size, tm.rank, q0, q1);
    double* V = I.V;
    double* btp = I.rhs;  // panel copy of the trailing part of Q^T b
    for (int e = tid; e < (q1 - q0) * kk; e += NT) {
      const int rr = q0 + e / kk, t = e - (e / kk) * kk;
      V[(size_t)rr * KM + t] = ldcg(Wcol(s_J[t]) + nP + rr);
    }
    for (int rr = q0 + tid; rr < q1; rr += NT) btp[rr] = ldcg(I.bt + nP + rr);
    __syncthreads();  // the dots below read rows other threads just copied
    __shared__ double s_sum[KM + 1];
    __shared__ double s_f[KM + 1];
    const int k0 = kk;
    int i = 0;
    for (; i < k0; ++i) {
      // partial dots over own rows r > i: column i with every panel column and b
      // (slots alternate with the parity of i: a fast CTA writing reflector
      // i+1 must not overwrite what a slow CTA still reads for reflector i)
      const int pb = (i & 1) * (KM + 1);
      for (int l = warp; l <= k0; l += NW) {
        double s = 0.0;
        for (int rr = max(q0, i + 1) + lane; rr < q1; rr += 32) {
          const double vi = ldcg(V + (size_t)rr * KM + i);
          const double y = (l < k0) ? ldcg(V + (size_t)rr * KM + l) : ldcg(btp + rr);
          s = fma(y, vi, s);
        }
        s = warp_sum(s);
        if (lane == 0) I.part[(size_t)tm.rank * PW + pb + l] = s;
      }
      if (!sync()) return false;
      {
        // two-level reduction of the team's partials: warp w sums the CTAs
        // t = w (mod NW), then the NW partial sums are added in order
        double* sR = dyn;  // NW x (KM + 1)
        for (int l = lane; l <= k0; l += 32) {
          double sacc = 0.0;
          for (int t = warp; t < tm.size; t += NW) sacc += ldcg(I.part + (size_t)t * PW + pb + l);
          sR[warp * (KM + 1) + l] = sacc;
        }
        __syncthreads();
        if (tid <= k0) {
          double sacc = 0.0;
          for (int w2 = 0; w2 < NW; ++w2) sacc += sR[w2 * (KM + 1) + tid];
          s_sum[tid] = sacc;
        }
        __syncthreads();
      }
      const double xii = ldcg(V + (size_t)i * KM + i);
      const double alpha = sqrt_gm(xii * xii + s_sum[i]);
      const double an = ldcg(I.anorm + s_J[i]);
      if (i >= L || !(alpha > (100.0 * EPS) * an)) break;
      const double sg = (xii >= 0.0) ? 1.0 : -1.0;
      const double v0 = xii + sg * alpha;
      const double beta = 2.0 * rcp_nr(v0 * v0 + s_sum[i]);
      if (tid <= k0) {
        double f = 0.0;
        if (tid > i && tid < k0) f = beta * (v0 * ldcg(V + (size_t)i * KM + tid) + s_sum[tid]);
        if (tid == k0) f = beta * (v0 * ldcg(btp + i) + s_sum[k0]);
        s_f[tid] = f;
      }
      __syncthreads();
      // rank 0 records R22 row i, the panel right-hand side, v0, beta, T
      if (tm.rank == 0) {
        if (tid == i) I.R22[i + i * KM] = -sg * alpha;
        if (tid > i && tid < k0) I.R22[i + tid * KM] = ldcg(V + (size_t)i * KM + tid) - s_f[tid] * v0;
        if (tid == k0) I.pr[i] = ldcg(btp + i) - s_f[k0] * v0;
        if (tid == 0) {
          I.vtop[i] = v0;
          I.beta[i] = beta;
          I.T[i + i * KM] = beta;
        }
        // T[0:i, i] = -beta T[0:i, 0:i] z,  z_s = v_s^T v_i
        __shared__ double s_z[KM];
        if (tid < i) s_z[tid] = ldcg(V + (size_t)i * KM + tid) * v0 + s_sum[tid];
        __syncthreads();
        if (tid < i) {
          double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
          int s = tid;
          for (; s + 3 < i; s += 4) {
            a0 = fma(ldcg(I.T + tid + s * KM), s_z[s], a0);
            a1 = fma(ldcg(I.T + tid + (s + 1) * KM), s_z[s + 1], a1);
            a2 = fma(ldcg(I.T + tid + (s + 2) * KM), s_z[s + 2], a2);
            a3 = fma(ldcg(I.T + tid + (s + 3) * KM), s_z[s + 3], a3);
          }
          for (; s < i; ++s) a0 = fma(ldcg(I.T + tid + s * KM), s_z[s], a0);
          I.T[tid + i * KM] = -beta * ((a0 + a1) + (a2 + a3));
        }
      }
      flops(PH_PANEL, 2.0 * (double)(2 * (k0 - i) + 1) * (double)(L - i));
      // update own rows r > i of the later columns and of b
      const int nl = k0 - i;  // columns i+1..k0-1 and b
      for (int e = tid; e < (q1 - max(q0, i + 1)) * nl; e += NT) {
        const int rr = max(q0, i + 1) + e / nl;
        const int l = i + 1 + (e - (e / nl) * nl);
        const double vi = ldcg(V + (size_t)rr * KM + i);
        if (l < k0) V[(size_t)rr * KM + l] = ldcg(V + (size_t)rr * KM + l) - s_f[l] * vi;
        else btp[rr] = ldcg(btp + rr) - s_f[k0] * vi;
      }
      __syncthreads();
    }
    kk = i;  // reflectors formed (truncated by the rank bound)
    if constexpr (std::is_same<Team, CtaTeam>::value) {
      // a one-CTA team holds every row: the digits of the tensor-core commit
      if (I.Vd != nullptr && kk > 4 && kk <= 32) {
        __syncthreads();
        for (int rr = warp; rr < L; rr += NW) {
          const double v0 = (lane < kk) ? ldcg(I.vtop + lane) : 1.0;
          const double vr = (lane < kk) ? (rr > lane ? ldcg(V + (size_t)rr * KM + lane) : (rr == lane ? v0 : 0.0)) : 0.0;
          vd_store_row(rr, vr, v0);
        }
        vd_ok = true;
      }
    }
    return sync();
  }

  // One row of the panel's reflectors as 7-bit digits for the tensor-core
  // commit (one warp; lane t holds V(row, t) - v0 on the diagonal, zero
  // above - and v0 of reflector t).  Reflector t is scaled by 2^-Ft,
  // 2^Ft > |v0| >= |V(:, t)|; the row scale is the largest exponent bound of
  // the scaled row, and even lanes store digit pairs.
  __device__ __forceinline__ void vd_store_row(int row, double vrow, double v0) {
    const double v = scale2(vrow, -ebound(v0));
    const int er = __reduce_max_sync(0xffffffffu, ebound(v));
    unsigned ha, la;
    halves28(fix56(v, 56 - er), ha, la);
    const unsigned hb = __shfl_down_sync(0xffffffffu, ha, 1), lb = __shfl_down_sync(0xffffffffu, la, 1);
    const bool nega = v < 0.0;
    const bool negb = __shfl_down_sync(0xffffffffu, nega ? 1 : 0, 1) != 0;
    unsigned sg, nb2;
    sign2(nega, negb, sg, nb2);
    if ((lane & 1) == 0) {
      // a row holds its ND digit planes (16 words each) side by side;
      // 16-byte chunk c of the row is stored at c ^ (row & 7), as the
      // commit's shared-memory layout expects
      const int w = lane >> 1;
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        const int c = (4 * k + (w >> 2)) ^ (row & 7);
        I.Vd[(size_t)row * (16 * ND) + c * 4 + (w & 3)] = dig2k(k, ha, la, hb, lb, sg, nb2);
      }
    }
    if (lane == 0) I.Ver[row] = er;
  }

  // Panel with the team's rows held in shared memory (at most PR_MAX rows
  // per CTA): the same Householder steps as panel(), one barrier per
  // reflector.  Each CTA keeps rows [q0, q1) of the kk selected columns and
  // of Q^T b (column kk) for the whole panel; per reflector i it adds its
  // dots into the team's fixed-point sums at L2 and, if it owns row i,
  // publishes the pivot row; after the barrier every CTA reads the sums
  // (no CTA adds the team's partials itself: one FP64 add is 64 cycles of
  // a sub-partition on this GPU, and every CTA would repeat them).  The scalars of
  // a reflector are formed once per CTA and shared; T is built by rank 0
  // after the last reflector from the saved products z_s = v_s^T v_i.
  // (FP64 issue is the scarce resource here: every warp instruction counts.)
  static constexpr int PR_MAX = 128;     // rows per CTA of the shared-memory panel
  static constexpr int PANEL_ROWS = 32;  // target rows per panel CTA
  static constexpr int PS = KM + 1;  // row stride of the staged panel
  __device__ bool panel_smem(const int* s_J, int P) {
    const int L = I.m - nP;
    if (kk > L) kk = L;
    if (tm.rank < P && !panel_rows(s_J, P, L)) return false;
    if (tm.rank == 0 && tid == 0) I.ctl[C_KK] = kk;
    if (!sync()) return false;
    tm.sub_reset();
    // every exchange sum is read: the next panel's first exchange adds into
    // buffer 0 again
    if (tm.rank == 0)
      for (int e = tid; e < PACC_W; e += NT) I.pacc[e] = 0;
    kk = ldcg(I.ctl + C_KK);
    vd_ok = I.Vd != nullptr && kk > 4 && kk <= 32;
    return true;
  }
  // The panel on ranks 0 .. P-1 (rows split over them), with the sub-team
  // barrier; kk is left at the number of reflectors formed.
  __device__ bool panel_rows(const int* s_J, int P, int L) {
    const int k0 = kk, NL = k0 + 1;
    int q0, q1;
    split(L, P, tm.rank, q0, q1);
    const int nr = q1 - q0;
    double* sP = dyn;                   // nr x PS: own rows, columns 0..k0 (k0 = Q^T b)
    double* sZ = dyn + PR_MAX * PS;     // KM x KM, rank 0: z_s of reflector i at sZ[s + i KM]
    double* sG = sZ + KM * KM;          // reduction scratch (2 NT doubles)
    double* sT = sG + 2 * NT;           // KM x KM, rank 0: T
    __shared__ double s_sum[KM + 1], s_f[KM + 1], s_piv[KM + 1], s_an[KM], s_bt[KM];
    __shared__ double s_k[KM + 1], s_piv2[KM + 1], s_xp[KM + 1], s_A[KM + 1], s_H[KM + 1], s_f2[KM + 1], s_g[KM + 1];
    __shared__ double s_sc[8];          // alpha, v0, beta, sign; the same for the second reflector
    __shared__ double s_v0[KM];         // v0 of every reflector (every CTA)
    __shared__ int s_stop, s_stop2;
    for (int e = tid; e < nr * NL; e += NT) {
      const int rr = e / NL, l = e - rr * NL;
      sP[rr * PS + l] = (l < k0) ? ldcg(Wcol(s_J[l]) + nP + q0 + rr) : ldcg(I.bt + nP + q0 + rr);
    }
    if (tid < k0) s_an[tid] = ldcg(I.anorm + s_J[tid]);
    // Exponent bounds of the panel columns' norms: u_j for a selected
    // column (its trailing norm; the reflectors are orthogonal, so no part
    // of the column below a pivot is longer) and ||b|| for Q^T b.  The dot
    // of panel columns l and l' over any rows is below 2^(s_ex[l] + s_ex[l']),
    // and half of that with the + 1 that the exchange adds.
    __shared__ int s_ex[KM + 1];
    if (tid < k0) s_ex[tid] = max(ebound(ldcg(I.u + s_J[tid])), -1000);
    if (tid == k0) s_ex[tid] = max(ebound(sqrt(bsq)), -1000);
    // The team's sums of an exchange are added up at L2 as fixed-point
    // integers in units of 2^-55 of that bound (exact and order-free, so
    // every run gives the same bits; the truncation of the P partials is
    // below P 2^-53 u_l u_l', FP64's own bound for adding them), into
    // buffer step mod 3, spread over PACC_COPIES copies to cut the
    // contention on each word; rank 0 zeroes the buffer of the next
    // exchange, whose previous readers all passed the barrier before this one.
    const bool solo = P == 1;  // one CTA: its own sums are the team's
    const int cp = (tm.rank % PACC_COPIES) * 2 * (KM + 1);
    __syncthreads();
    // owner of a panel row: the rank whose split range holds it
    auto owner = [&](int row) {
      int r = (int)(((long long)row * P) / max(L, 1));
      int lo, hi;
      for (;;) {
        split(L, P, r, lo, hi);
        if (row < lo) --r;
        else if (row >= hi) ++r;
        else return r;
      }
    };
    // owners of the pivot rows 0 .. k0-1 (k0 <= L), once per panel
    __shared__ int s_own[KM];
    if (tid < k0) s_own[tid] = owner(tid);
    __syncthreads();
    // thread (gl, gg): column gl, group gg of G
    const int G = NT / NL, gl = tid % NL, gg = tid / NL;
    const bool actg = gg < G;
    int i = 0;
    int step = 0;  // exchanges so far (parity of the partial-sum slots)
    bool stopped = false;
    // Reflectors two at a time, one exchange for both.  With x the columns
    // before reflector i (rows > i), the exchange carries G_l = x_i^T x_l
    // (rows > i), K_l = x_{i+1}^T x_l (rows > i+1) and pivot rows i and
    // i+1.  Reflector i is formed as in the single step; then, with
    // A_l = x_i^T x_l and B = x_i^T x_i over rows > i+1, the columns after
    // reflector i satisfy x'_{i+1}^T x'_l = K_l - f_l A_{i+1} - f_{i+1} A_l
    // + f_{i+1} f_l B (A_{i+1} = K_i) and x'_l[i+1] = x_l[i+1] - f_l x_i[i+1],
    // which is all reflector i+1 needs.  Exact in exact arithmetic; the
    // rounding is of the order of the direct dots'.
    for (; i + 1 < k0; i += 2) {
      const int pb = (step & 1) * 4 * (KM + 1);
      long long* acc = I.pacc + (step % 3) * PACC_W;
      long long* acc_next = I.pacc + ((step + 1) % 3) * PACC_W;
      ++step;
      double* mypart = I.part + (size_t)tm.rank * PW;
      const int r0 = max(q0, i + 1) - q0, r1 = max(q0, i + 2) - q0;
      {
        double sg_ = 0.0, sk_ = 0.0;
        if (actg) {
          for (int rr = r0 + gg; rr < nr; rr += G) {
            const double xl = sP[rr * PS + gl];
            sg_ = fma(xl, sP[rr * PS + i], sg_);
            if (rr >= r1) sk_ = fma(xl, sP[rr * PS + i + 1], sk_);
          }
          sG[gg * NL + gl] = sg_;
          sG[NT + gg * NL + gl] = sk_;
        }
        __syncthreads();
        for (int st = 1; st < G; st <<= 1) {
          if (actg && (gg & (2 * st - 1)) == 0 && gg + st < G) {
            sG[gg * NL + gl] += sG[(gg + st) * NL + gl];
            sG[NT + gg * NL + gl] += sG[NT + (gg + st) * NL + gl];
          }
          __syncthreads();
        }
        if (!solo && tid <= k0) {
          atomicAdd(reinterpret_cast<unsigned long long*>(acc + cp + tid),
                    (unsigned long long)fx_q(sG[tid], s_ex[i] + s_ex[tid] + 1));
          atomicAdd(reinterpret_cast<unsigned long long*>(acc + cp + (KM + 1) + tid),
                    (unsigned long long)fx_q(sG[NT + tid], s_ex[i + 1] + s_ex[tid] + 1));
        }
        if (!solo && tm.rank == 0)
          for (int e = tid; e < PACC_W; e += NT) acc_next[e] = 0;
      }
      if (i >= q0 && i < q1 && tid <= k0) mypart[pb + 2 * (KM + 1) + tid] = sP[(i - q0) * PS + tid];
      if (i + 1 >= q0 && i + 1 < q1 && tid <= k0) mypart[pb + 3 * (KM + 1) + tid] = sP[(i + 1 - q0) * PS + tid];
      if (!tm.sync_sub(P)) return false;
      {
        const int own = s_own[i], own2 = s_own[i + 1];
        if (tid <= k0) {
          s_piv[tid] = ldcg(I.part + (size_t)own * PW + pb + 2 * (KM + 1) + tid);
          s_piv2[tid] = ldcg(I.part + (size_t)own2 * PW + pb + 3 * (KM + 1) + tid);
        }
        if (!solo && tid <= k0) {
          long long qg = 0, qk = 0;
#pragma unroll
          for (int c = 0; c < PACC_COPIES; ++c) {
            qg += __ldcg(acc + c * 2 * (KM + 1) + tid);
            qk += __ldcg(acc + c * 2 * (KM + 1) + (KM + 1) + tid);
          }
          sG[tid] = fx_x(qg, s_ex[i] + s_ex[tid] + 1);
          sG[NT + tid] = fx_x(qk, s_ex[i + 1] + s_ex[tid] + 1);
        }
        __syncthreads();
      }
      // reflector i
      if (warp == 0 && lane == 0) {
        const double xii = s_piv[i], ssum_i = sG[i];
        const double alpha = sqrt_gm(fma(xii, xii, ssum_i));
        const int stop = (i >= L || !(alpha > (100.0 * EPS) * s_an[i])) ? 1 : 0;
        const double sg = (xii >= 0.0) ? 1.0 : -1.0;
        const double v0 = xii + sg * alpha;
        s_stop = stop;
        s_sc[0] = alpha;
        s_sc[1] = v0;
        s_sc[2] = stop ? 0.0 : 2.0 * rcp_nr(fma(v0, v0, ssum_i));
        s_sc[3] = sg;
      }
      __syncthreads();
      if (s_stop) {
        stopped = true;
        break;
      }
      const double v0 = s_sc[1], beta = s_sc[2];
      if (tid == 0) s_v0[i] = v0;
      if (tid <= k0) {
        const double gs = sG[tid], ks = sG[NT + tid];
        s_sum[tid] = gs;
        s_k[tid] = ks;
        const double f = (tid > i) ? beta * fma(v0, s_piv[tid], gs) : 0.0;
        s_f[tid] = f;
        // row i+1 after reflector i, and A_l over rows > i+1
        s_xp[tid] = fma(-f, s_piv2[i], s_piv2[tid]);
        s_A[tid] = fma(-s_piv2[i], s_piv2[tid], gs);
      }
      __syncthreads();
      if (tid <= k0) {
        const double fi1 = s_f[i + 1], Ai1 = s_k[i];
        const double Bq = fma(-s_piv2[i], s_piv2[i], s_sum[i]);
        const double fl = s_f[tid];
        double h = fma(-fl, Ai1, s_k[tid]);
        h = fma(-fi1, s_A[tid], h);
        h = fma(fi1 * fl, Bq, h);
        s_H[tid] = h;
      }
      __syncthreads();
      // reflector i+1 on the columns after reflector i
      if (warp == 0 && lane == 0) {
        const double xii = s_xp[i + 1], ssum_i = s_H[i + 1];
        const double alpha = sqrt_gm(fma(xii, xii, ssum_i));
        const int stop = (i + 1 >= L || !(alpha > (100.0 * EPS) * s_an[i + 1])) ? 1 : 0;
        const double sg = (xii >= 0.0) ? 1.0 : -1.0;
        const double v0b = xii + sg * alpha;
        s_stop2 = stop;
        s_sc[4] = alpha;
        s_sc[5] = v0b;
        s_sc[6] = stop ? 0.0 : 2.0 * rcp_nr(fma(v0b, v0b, ssum_i));
        s_sc[7] = sg;
      }
      __syncthreads();
      const bool two = !s_stop2;
      const double v0b = s_sc[5], beta2 = s_sc[6];
      if (tid == 0 && two) s_v0[i + 1] = v0b;
      if (tid <= k0) {
        s_f2[tid] = (two && tid > i + 1) ? beta2 * fma(v0b, s_xp[tid], s_H[tid]) : 0.0;
        s_g[tid] = fma(-s_f2[tid], s_f[i + 1], s_f[tid]);
        if (tm.rank == 0 && tid < i) sZ[tid + i * KM] = fma(s_piv[tid], v0, s_sum[tid]);  // z_s = v_s^T v_i
        if (tm.rank == 0 && two && tid <= i) {
          // z_s = v_s^T v_{i+1}: v_s[i+1] v0' + x_s^T x'_{i+1} over rows > i+1
          const double xs_x = (tid == i) ? fma(-s_f[i + 1], fma(-s_piv2[i], s_piv2[i], s_sum[i]), s_k[i])
                                         : fma(-s_f[i + 1], s_A[tid], s_k[tid]);
          sZ[tid + (i + 1) * KM] = fma(s_piv2[tid], v0b, xs_x);
        }
      }
      __syncthreads();
      if (tm.rank == 0) {
        if (tid == i) I.R22[i + i * KM] = -s_sc[3] * s_sc[0];
        if (tid > i && tid < k0) I.R22[i + tid * KM] = s_piv[tid] - s_f[tid] * v0;
        if (tid == k0) I.pr[i] = s_piv[k0] - s_f[k0] * v0;
        if (tid == 0) {
          I.vtop[i] = v0;
          I.beta[i] = beta;
          s_bt[i] = beta;
        }
        if (two) {
          if (tid == i + 1) I.R22[(i + 1) + (i + 1) * KM] = -s_sc[7] * s_sc[4];
          if (tid > i + 1 && tid < k0) I.R22[(i + 1) + tid * KM] = s_xp[tid] - s_f2[tid] * v0b;
          if (tid == k0) I.pr[i + 1] = s_xp[k0] - s_f2[k0] * v0b;
          if (tid == 0) {
            I.vtop[i + 1] = v0b;
            I.beta[i + 1] = beta2;
            s_bt[i + 1] = beta2;
          }
        }
      }
      flops(PH_PANEL, 2.0 * (double)(2 * (k0 - i) + 1) * (double)(L - i));
      if (two) flops(PH_PANEL, 2.0 * (double)(2 * (k0 - i - 1) + 1) * (double)(L - i - 1));
      // own rows: reflector i on rows > i (columns > i), then reflector i+1
      // on rows > i+1 (columns > i+1), both in two FMAs per element from
      // the row's columns i and i+1 before either reflector (columns i+2 ..
      // first, reading column i+1 before it is updated)
      {
        const int nl = k0 - i - 1;
        for (int e = tid; e < (nr - r0) * nl; e += NT) {
          const int rr = r0 + e / nl, l = i + 2 + (e - (e / nl) * nl);
          const double xi = sP[rr * PS + i];
          double x;
          if (two && rr >= r1) {
            // x - f_l x_i - f2_l (x_{i+1} - f_{i+1} x_i), with g_l = f_l - f2_l f_{i+1}
            x = fma(-s_g[l], xi, sP[rr * PS + l]);
            x = fma(-s_f2[l], sP[rr * PS + i + 1], x);
          } else {
            x = fma(-s_f[l], xi, sP[rr * PS + l]);
          }
          sP[rr * PS + l] = x;
        }
      }
      __syncthreads();
      for (int rr = r0 + tid; rr < nr; rr += NT)
        sP[rr * PS + i + 1] = fma(-s_f[i + 1], sP[rr * PS + i], sP[rr * PS + i + 1]);
      __syncthreads();
      if (!two) {
        i += 1;
        stopped = true;
        break;
      }
    }
    for (; i < k0 && !stopped; ++i) {
      const int pb = (step & 1) * 4 * (KM + 1);
      long long* acc = I.pacc + (step % 3) * PACC_W;
      long long* acc_next = I.pacc + ((step + 1) % 3) * PACC_W;
      ++step;
      double* mypart = I.part + (size_t)tm.rank * PW;
      // dots of column i with every column (and Q^T b) over own rows > i:
      // rows r0 + gg, r0 + gg + G, ... per thread, then a pairwise tree
      const int r0 = max(q0, i + 1) - q0;
      {
        double sacc = 0.0;
        if (actg)
          for (int rr = r0 + gg; rr < nr; rr += G) sacc = fma(sP[rr * PS + gl], sP[rr * PS + i], sacc);
        if (actg) sG[gg * NL + gl] = sacc;
        __syncthreads();
        for (int st = 1; st < G; st <<= 1) {
          if (actg && (gg & (2 * st - 1)) == 0 && gg + st < G) sG[gg * NL + gl] += sG[(gg + st) * NL + gl];
          __syncthreads();
        }
        if (!solo && tid <= k0)
          atomicAdd(reinterpret_cast<unsigned long long*>(acc + cp + tid),
                    (unsigned long long)fx_q(sG[tid], s_ex[i] + s_ex[tid] + 1));
        if (!solo && tm.rank == 0)
          for (int e = tid; e < PACC_W; e += NT) acc_next[e] = 0;
      }
      if (i >= q0 && i < q1 && tid <= k0) mypart[2 * (KM + 1) + pb + tid] = sP[(i - q0) * PS + tid];
      if (!tm.sync_sub(P)) return false;
      // the team's dots from the fixed-point sums; the pivot row from its owner
      {
        const int own = s_own[i];
        if (tid <= k0) s_piv[tid] = ldcg(I.part + (size_t)own * PW + 2 * (KM + 1) + pb + tid);
        if (!solo && tid <= k0) {
          long long qg = 0;
#pragma unroll
          for (int c = 0; c < PACC_COPIES; ++c) qg += __ldcg(acc + c * 2 * (KM + 1) + tid);
          sG[tid] = fx_x(qg, s_ex[i] + s_ex[tid] + 1);
        }
        __syncthreads();
      }
      // the reflector's scalars, once per CTA (warp 0), and f for every column
      if (warp == 0) {
        const double ssum_i = sG[i];
        if (lane == 0) {
          const double xii = s_piv[i];
          const double alpha = sqrt_gm(fma(xii, xii, ssum_i));
          const int stop = (i >= L || !(alpha > (100.0 * EPS) * s_an[i])) ? 1 : 0;
          const double sg = (xii >= 0.0) ? 1.0 : -1.0;
          const double v0 = xii + sg * alpha;
          s_stop = stop;
          s_sc[0] = alpha;
          s_sc[1] = v0;
          s_sc[2] = stop ? 0.0 : 2.0 * rcp_nr(fma(v0, v0, ssum_i));
          s_sc[3] = sg;
        }
      }
      __syncthreads();
      if (s_stop) break;
      const double v0 = s_sc[1], beta = s_sc[2];
      if (tid == 0) s_v0[i] = v0;
      if (tid <= k0) {
        const double ssum = sG[tid];
        s_sum[tid] = ssum;
        s_f[tid] = (tid > i) ? beta * fma(v0, s_piv[tid], ssum) : 0.0;
        if (tm.rank == 0 && tid < i) sZ[tid + i * KM] = fma(s_piv[tid], v0, ssum);  // z_s = v_s^T v_i
      }
      __syncthreads();
      if (tm.rank == 0) {
        if (tid == i) I.R22[i + i * KM] = -s_sc[3] * s_sc[0];
        if (tid > i && tid < k0) I.R22[i + tid * KM] = s_piv[tid] - s_f[tid] * v0;
        if (tid == k0) I.pr[i] = s_piv[k0] - s_f[k0] * v0;
        if (tid == 0) {
          I.vtop[i] = v0;
          I.beta[i] = beta;
          s_bt[i] = beta;
        }
      }
      flops(PH_PANEL, 2.0 * (double)(2 * (k0 - i) + 1) * (double)(L - i));
      // update own rows > i of the later columns and of Q^T b
      const int nl = k0 - i;
      for (int e = tid; e < (nr - r0) * nl; e += NT) {
        const int rr = r0 + e / nl, l = i + 1 + (e - (e / nl) * nl);
        sP[rr * PS + l] = fma(-s_f[l], sP[rr * PS + i], sP[rr * PS + l]);
      }
      __syncthreads();
    }
    kk = i;  // reflectors formed (truncated by the rank bound)
    // V rows of this CTA (reflector components below the diagonal)
    for (int e = tid; e < nr * kk; e += NT) {
      const int rr = e / kk, t = e - rr * kk;
      I.V[(size_t)(q0 + rr) * KM + t] = sP[rr * PS + t];
    }
    // the same rows as 7-bit digits for the tensor-core commit
    if (I.Vd != nullptr && kk > 4 && kk <= 32) {
      for (int rr = warp; rr < nr; rr += NW) {
        const int row = q0 + rr;
        vd_store_row(row, (lane < kk) ? (row > lane ? sP[rr * PS + lane] : (row == lane ? s_v0[lane] : 0.0)) : 0.0,
                     (lane < kk) ? s_v0[lane] : 1.0);
      }
    }
    if (tm.rank == 0) {
      // T is the inverse of the upper triangle M with M[r][r] = 1/beta_r and
      // M[r][s] = z_rs = v_r^T v_s (r < s).  Column c by back substitution on
      // one warp, all columns at once: x[c] = beta_c, then for s = c .. 1 the
      // lanes add z_rs x[s] into row r < s and x[s-1] = -beta_{s-1} acc[s-1]
      // (lane r holds rows r and r + 32; sT column-major with stride KM).
      for (int c = warp; c < kk; c += NW) {
        double acc0 = 0.0, acc1 = 0.0;
        double xs = s_bt[c];
        if (lane == 0) sT[c + c * KM] = xs;
        for (int sidx = c; sidx >= 1; --sidx) {
          if (lane < sidx) acc0 = fma(sZ[lane + sidx * KM], xs, acc0);
          if (lane + 32 < sidx) acc1 = fma(sZ[lane + 32 + sidx * KM], xs, acc1);
          const int r = sidx - 1;
          const double a = __shfl_sync(0xffffffffu, r < 32 ? acc0 : acc1, r & 31);
          xs = -s_bt[r] * a;
          if (lane == 0) sT[r + c * KM] = xs;
        }
      }
      __syncthreads();
      for (int e = tid; e < kk * kk; e += NT) {
        const int c = e / kk, r = e - c * kk;
        if (r <= c) I.T[r + c * KM] = sT[r + c * KM];
      }
    }
    return true;
  }

  // Back substitution with the kk x kk triangle R22 (one warp).
  __device__ void solve_r22(int k, double* y) {
    double a0 = (lane < k) ? ldcg(I.pr + lane) : 0.0;
    double a1 = (lane + 32 < k) ? ldcg(I.pr + lane + 32) : 0.0;
    // reciprocal diagonal computed by all lanes at once, off the chain
    const double r0 = (lane < k) ? rcp_nr(ldcg(I.R22 + lane + lane * KM)) : 0.0;
    const double r1 = (lane + 32 < k) ? rcp_nr(ldcg(I.R22 + (lane + 32) + (lane + 32) * KM)) : 0.0;
    double y0 = 0.0, y1 = 0.0;
    for (int jj = k - 1; jj >= 0; --jj) {
      const int owner = jj & 31;
      const bool hi = jj >= 32;
      double yv = 0.0;
      if (lane == owner) yv = (hi ? a1 : a0) * (hi ? r1 : r0);
      yv = __shfl_sync(0xffffffffu, yv, owner);
      if (lane == owner) { if (hi) y1 = yv; else y0 = yv; }
      if (lane < jj) a0 -= ldcg(I.R22 + lane + jj * KM) * yv;
      if (lane + 32 < jj) a1 -= ldcg(I.R22 + lane + 32 + jj * KM) * yv;
    }
    if (lane < k) y[lane] = y0;
    if (lane + 32 < k) y[lane + 32] = y1;
  }

  // Feasibility loop of Algorithm 3: drop the last J column while
  // min y_J <= 0 (and |J| > 1).  y_J only depends on the R22 triangle.  With
  // the positivity trick a J column enters with the sign of its w, and its y
  // in [A -A] is that sign times the physical y.
  __device__ bool feasibility(const int* s_J) {
    if (tm.rank == 0 && warp == 0) {
      __shared__ double s_y[KM];
      int k = kk, drops = 0;
      for (;;) {
        solve_r22(k, s_y);
        __syncwarp();
        double mn = INFINITY;
        for (int t = lane; t < k; t += 32) {
          const double sg = (sgn && ldcg(I.w + s_J[t]) < 0.0) ? -1.0 : 1.0;
          mn = fmin(mn, sg * s_y[t]);
        }
        mn = warp_max(-mn);
        mn = -mn;
        if (!(mn <= 0.0) || k <= 1) break;
        --k;
        ++drops;
      }
      for (int t = lane; t < k; t += 32) I.yJ[t] = s_y[t];
      if (lane == 0) {
        I.ctl[C_KP] = k;
        I.ctl[C_DROPS] = drops;
      }
    }
    if (!sync()) return false;
    kp = ldcg(I.ctl + C_KP);
    n_drop += ldcg(I.ctl + C_DROPS);
    return true;
  }

  // ------------------------------------------------------------ triangular solve
  // R y = rhs on positions [0, np) (the back substitution of subproblem (6));
  // y lands in yP.  Teams of several CTAs with more than two TB-blocks take
  // the flag-pipelined solve, everything else the blocked solve.
  __device__ bool trsv(int np) {
    if (np <= 0) return true;
    flops(cur_phase < 0 ? PH_SOLVE : cur_phase, (double)np * np);
    if (I.Dinv && tm.size >= 2 && np > 2 * TB) return trsv_pipelined(np);
    return trsv_blocked(np);
  }

  // Blocked back substitution, one team barrier per TB-block.  Rank 0 solves
  // each diagonal block from shared memory (staged in parallel) after folding
  // in the block just solved; the other rows receive that block's
  // contribution spread over the whole team.  rhs is consumed.
  __device__ bool trsv_blocked(int np) {
    const int nb = (np + TB - 1) / TB;
    __shared__ double s_y[TB];
    __shared__ int s_slot[TB];
    double* sD = dyn;                   // TB x (TB+1): sD[col * (TB+1) + row]
    double* sP = dyn + TB * (TB + 1);   // 8 x TB partial contributions
    for (int bi = nb - 1; bi >= 0; --bi) {
      const int b0 = bi * TB, b1 = min(np, b0 + TB), nbk = b1 - b0;
      const bool has_next = bi + 1 < nb;
      const int c0 = b0 + TB, c1 = min(np, c0 + TB), nc = c1 - c0;
      if (has_next && tid < nc) {
        s_y[tid] = ldcg(I.yP + c0 + tid);
        s_slot[tid] = ldcg(I.rslot + c0 + tid);
      }
      __syncthreads();
      if (has_next) {
        if constexpr (std::is_same<Team, CtaTeam>::value) {
          // one CTA: a thread per row, over the block's columns (loads of a
          // column coalesced across the rows; no cross-lane sums, which cost
          // five FP64 instructions per row and warp)
          for (int row = tid; row < b0; row += NT) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int j = 0;
            for (; j + 3 < nc; j += 4) {
              a0 = fma(ldcg(Rcol(s_slot[j]) + row), s_y[j], a0);
              a1 = fma(ldcg(Rcol(s_slot[j + 1]) + row), s_y[j + 1], a1);
              a2 = fma(ldcg(Rcol(s_slot[j + 2]) + row), s_y[j + 2], a2);
              a3 = fma(ldcg(Rcol(s_slot[j + 3]) + row), s_y[j + 3], a3);
            }
            for (; j < nc; ++j) a0 = fma(ldcg(Rcol(s_slot[j]) + row), s_y[j], a0);
            I.rhs[row] = ldcg(I.rhs + row) - ((a0 + a1) + (a2 + a3));
          }
        } else {
          // rows [0, b0): contribution of block bi+1, one warp per row
          // (lanes over the block's columns: all loads independent), rows
          // spread over the team
          const int gw = tm.rank * NW + warp, nwt = tm.size * NW;
          for (int row = gw; row < b0; row += nwt) {
            const double p0 = (lane < nc) ? ldcg(Rcol(s_slot[lane]) + row) * s_y[lane] : 0.0;
            const double p1 = (lane + 32 < nc) ? ldcg(Rcol(s_slot[lane + 32]) + row) * s_y[lane + 32] : 0.0;
            const double sacc = warp_sum(p0 + p1);
            if (lane == 0) I.rhs[row] = ldcg(I.rhs + row) - sacc;
          }
        }
      }
      if (tm.rank == 0) {
        // stage the diagonal block (upper triangle), its reciprocal diagonal
        // and the partial contributions of block bi+1 to rows [b0, b1)
        __shared__ int s_bslot[TB];
        __shared__ double s_rinv[TB];
        if (tid < nbk) s_bslot[tid] = ldcg(I.rslot + b0 + tid);
        __syncthreads();
        {
          double v[TB * TB / NT];
#pragma unroll
          for (int q2 = 0; q2 < TB * TB / NT; ++q2) {
            const int idx = tid + q2 * NT, cl = idx / TB, rw = idx - cl * TB;
            v[q2] = (cl < nbk && rw <= cl) ? ldcg(Rcol(s_bslot[cl]) + b0 + rw) : 0.0;
          }
#pragma unroll
          for (int q2 = 0; q2 < TB * TB / NT; ++q2) {
            const int idx = tid + q2 * NT, cl = idx / TB, rw = idx - cl * TB;
            sD[cl * (TB + 1) + rw] = v[q2];
            if (rw == cl && cl < nbk) s_rinv[cl] = rcp_nr(v[q2]);
          }
        }
        if (has_next) {
          const int rw = tid & (TB - 1), g = tid / TB;  // 8 groups of TB/8 columns
          double v[TB / 8];
#pragma unroll
          for (int q2 = 0; q2 < TB / 8; ++q2) {
            const int j = g * (TB / 8) + q2;
            v[q2] = (rw < nbk && j < nc) ? ldcg(Rcol(s_slot[j]) + b0 + rw) : 0.0;
          }
          double sacc = 0.0;
#pragma unroll
          for (int q2 = 0; q2 < TB / 8; ++q2) {
            const int j = g * (TB / 8) + q2;
            if (j < nc) sacc = fma(v[q2], s_y[j], sacc);
          }
          sP[g * TB + rw] = sacc;
        }
        __syncthreads();
        // columns scaled by their reciprocal diagonal: the substitution below
        // then needs no multiply on its chain (y_j = a_j / R_jj is formed for
        // every row at the end)
        for (int idx = tid; idx < TB * TB; idx += NT) {
          const int cl = idx / TB, rw = idx - cl * TB;
          if (cl < nbk && rw < cl) sD[cl * (TB + 1) + rw] *= s_rinv[cl];
        }
        __syncthreads();
        if (warp == 0) {
          double a0 = 0.0, a1 = 0.0;
          if (lane < nbk) {
            a0 = ldcg(I.rhs + b0 + lane);
            if (has_next)
              for (int g = 0; g < 8; ++g) a0 -= sP[g * TB + lane];
          }
          if (lane + 32 < nbk) {
            a1 = ldcg(I.rhs + b0 + lane + 32);
            if (has_next)
              for (int g = 0; g < 8; ++g) a1 -= sP[g * TB + lane + 32];
          }
          // a_i -= (R_ij / R_jj) a_j, j from the last row up; rows 32 .. 63
          // first (they feed both halves), then rows 0 .. 31 (one FMA a step)
          for (int jj = nbk - 1; jj >= 32; --jj) {
            const double* cj = sD + jj * (TB + 1);
            const double aj = __shfl_sync(0xffffffffu, a1, jj & 31);
            a0 = fma(-cj[lane], aj, a0);
            if (lane + 32 < jj) a1 = fma(-cj[lane + 32], aj, a1);
          }
          for (int jj = min(nbk, 32) - 1; jj >= 0; --jj) {
            const double* cj = sD + jj * (TB + 1);
            const double aj = __shfl_sync(0xffffffffu, a0, jj);
            if (lane < jj) a0 = fma(-cj[lane], aj, a0);
          }
          if (lane < nbk) I.yP[b0 + lane] = a0 * s_rinv[lane];
          if (lane + 32 < nbk) I.yP[b0 + lane + 32] = a1 * s_rinv[lane + 32];
        }
      }
      if (!sync()) return false;
    }
    return true;
  }


  // Flag-pipelined back substitution (teams of several CTAs).  Positions are
  // cut into TB-blocks; rank 0 walks them from the last to the first and is
  // the only CTA on the dependency chain.  For block b with right-hand side
  // a_b = rhs_b - R(b, b+1) y_{b+1} - acc_b it forms y_b = D_b^{-1} a_b with
  // the inverse of the diagonal block D_b kept from earlier solves, and back
  // substitution for the columns whose inverse is stale.  acc_b, the blocks
  // b+2, b+3, ... of the row block, is accumulated by ranks 1, 2, ... in
  // SLAB-row slabs as soon as each y block is published (a flag per block)
  // and handed back through a flag per slab.  The last ranks compute the
  // stale inverse columns meanwhile, for the solves that follow.  Column j of
  // the inverse of an upper triangular block depends only on the block's
  // leading (j+1) x (j+1) part, so appending positions leaves every computed
  // column valid; a deletion at position q invalidates positions >= q.
  __device__ bool trsv_pipelined(int np) {
    const int nb = (np + TB - 1) / TB;
    const int ep = ++tepoch;
    bool ok = true;
    if (tm.rank == 0) {
      ok = tri_chain(np, nb, ep);
    } else {
      // inverse columns first (they wait for nothing; rank 0 may wait for
      // them), then the slab accumulations
      tri_inverse(np, nb, ep);
      ok = tri_slabs(np, nb, ep);
    }
    if (!ok) {
      failed = true;
      status = LHDM_ERR_TIMEOUT;
      return false;
    }
    if (!sync()) return false;
    inv_valid = np;
    return true;
  }

  __device__ __forceinline__ int* yflags() const { return I.tflag; }
  __device__ __forceinline__ int* sflags() const { return I.tflag + (I.cap + TB - 1) / TB; }
  __device__ __forceinline__ int* iflags() const { return I.tflag + (1 + TB / SLAB) * ((I.cap + TB - 1) / TB); }

  // Rank 0: the chain over the blocks (see trsv_pipelined).  What a block
  // reads without waiting for y - its slots, the tile R(b, b+1), the
  // inverse columns cached by earlier solves and rhs - is copied to shared
  // memory (cp.async) while the block before it in the chain (b + 1)
  // finishes, so that a block waits only for the slab sums.
  __device__ bool tri_chain(int np, int nb, int ep) {
    double* sD = dyn;                       // TB x (TB+1) stale diagonal columns
    double* sP = dyn + TB * (TB + 1);       // 8 x TB partial sums
    double* sRT = sP + 8 * TB;              // TB x TB: R(b, b+1), column j at j TB
    double* sDI = sRT + TB * TB;            // TB x TB: the cached inverse columns
    __shared__ double s_rh[TB];
    __shared__ double s_a[TB];
    __shared__ double s_y[2][TB];
    __shared__ double s_rinv[TB];
    __shared__ int s_slot[2][TB];           // slots of block bi in s_slot[bi & 1]
    const int row = tid & (TB - 1), g = tid >> 6;  // 8 groups of 8 columns
    int* yfl = yflags();
    const int* ifl = iflags();
    int pslot = 0;
    double pacc = 0.0;  // the block's slab sum as last seen (ACC_EMPTY: not yet written)
    auto valid_cols = [&](int b0, int nbk) { return min(max(inv_valid - b0, 0), nbk); };
    // block bi's loads that wait for nothing (its columns' slots are those
    // of block bi + 1, already in s_slot)
    auto prefetch = [&](int bi) {
      const int b0 = bi * TB, nbk = min(np, b0 + TB) - b0;
      const int nc = (bi + 1 < nb) ? min(np, b0 + 2 * TB) - (b0 + TB) : 0;
      const int v = valid_cols(b0, nbk);
      const int* cs = s_slot[(bi + 1) & 1];
      pslot = (tid < nbk) ? ldcg(I.rslot + b0 + tid) : 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = g * 8 + q;
        const bool okr = row < nbk && j < nc, okd = row <= j && j < v;
        cp8(sRT + j * TB + row, okr ? Rcol(cs[j]) + b0 + row : I.rhs, okr);
        cp8(sDI + j * TB + row, okd ? I.Dinv + (size_t)bi * TB * TB + (size_t)j * TB + row : I.rhs, okd);
      }
      if (g == 0) cp8(s_rh + row, row < nbk ? I.rhs + b0 + row : I.rhs, row < nbk);
      cp_commit();
      if (g == 0 && row < nbk && bi + 2 < nb) pacc = ldcg(I.accb + b0 + row);
    };
    prefetch(nb - 1);
    for (int bi = nb - 1; bi >= 0; --bi) {
      const int b0 = bi * TB, nbk = min(np, b0 + TB) - b0;
      const int nc = (bi + 1 < nb) ? min(np, b0 + 2 * TB) - (b0 + TB) : 0;
      int v = valid_cols(b0, nbk);  // columns with a valid inverse
      double* ycur = s_y[bi & 1];
      const double* ynext = s_y[(bi + 1) & 1];
      int* s_bslot = s_slot[bi & 1];
      if (tid < nbk) s_bslot[tid] = pslot;
      cp_wait_all();  // this thread's copies of the block's operands
      if (bi < nb - 1 && v < nbk) {
        // the stale columns of this block are being inverted by the last
        // ranks in this call: wait for them instead of substituting, then
        // read the whole block's inverse
        int okw = 1;
        if (tid < INV_PARTS) okw = wait_ge(ifl + bi * INV_PARTS + tid, ep, tm_err(), I.wait_ns) ? 1 : 0;
        if (!__syncthreads_and(okw)) return false;
        v = nbk;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = g * 8 + q;
          sDI[j * TB + row] = (row <= j) ? ldcg(I.Dinv + (size_t)bi * TB * TB + (size_t)j * TB + row) : 0.0;
        }
      } else {
        __syncthreads();
      }
      if (v < nbk) {
        // stale columns of the diagonal block
        const int ns = (nbk - v) * TB;  // <= TB * TB = 8 per thread
        double sv[TB * TB / NT];
#pragma unroll
        for (int k = 0; k < TB * TB / NT; ++k) {
          const int idx = tid + k * NT, j = v + idx / TB, i = idx & (TB - 1);
          sv[k] = (idx < ns && i <= j) ? ldcg(Rcol(s_bslot[j]) + b0 + i) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < TB * TB / NT; ++k) {
          const int idx = tid + k * NT, j = v + idx / TB, i = idx & (TB - 1);
          if (idx < ns) {
            sD[j * (TB + 1) + i] = sv[k];
            if (i == j) s_rinv[j] = rcp_nr(sv[k]);
          }
        }
      }
      // contribution of block b+1 (just solved) to this block's rows
      if (nc > 0) {
        double p0 = 0.0, p1 = 0.0;
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          p0 = fma(sRT[(g * 8 + q) * TB + row], ynext[g * 8 + q], p0);
          p1 = fma(sRT[(g * 8 + q + 1) * TB + row], ynext[g * 8 + q + 1], p1);
        }
        sP[g * TB + row] = p0 + p1;
      }
      // slab accumulations of blocks b+2, ...: the value is its own flag
      // (written once per solve, 8-byte single-copy atomic), usually already
      // there when the block before this one read it ahead
      int okw = 1;
      double acc = 0.0;
      if (g == 0 && row < nbk && bi + 2 < nb) {
        acc = pacc;
        if (__double_as_longlong(acc) == ACC_EMPTY) {
          const long long tw0 = gtimer();
          unsigned spins = 0;
          for (;;) {
            acc = *(volatile const double*)(I.accb + b0 + row);
            if (__double_as_longlong(acc) != ACC_EMPTY) break;
            if ((++spins & 63u) == 0u) {
              int* er = tm_err();
              if ((er && *(volatile int*)er) || gtimer() - tw0 > I.wait_ns) {
                if (er) atomicExch(er, 1);
                okw = 0;
                break;
              }
            }
          }
        }
        I.accb[b0 + row] = __longlong_as_double(ACC_EMPTY);  // empty again for the next solve
      }
      if (!__syncthreads_and(okw)) return false;
      if (g == 0 && row < nbk) {
        double a = s_rh[row] - acc;
        if (nc > 0) {
          const double s01 = sP[row] + sP[TB + row], s23 = sP[2 * TB + row] + sP[3 * TB + row];
          const double s45 = sP[4 * TB + row] + sP[5 * TB + row], s67 = sP[6 * TB + row] + sP[7 * TB + row];
          a -= (s01 + s23) + (s45 + s67);
        }
        s_a[row] = a;
      }
      __syncthreads();
      if (v < nbk) {
        // back substitution over the stale columns [v, nbk); the rows
        // above v receive their contributions on the way
        if (warp == 0) {
          double a0 = (lane < nbk) ? s_a[lane] : 0.0;
          double a1 = (lane + 32 < nbk) ? s_a[lane + 32] : 0.0;
          for (int l = nbk - 1; l >= v; --l) {
            const int own = l & 31;
            const double* cl = sD + l * (TB + 1);
            double yv = (l >= 32 ? a1 : a0) * s_rinv[l];
            yv = __shfl_sync(0xffffffffu, yv, own);
            if (lane == own) ycur[l] = yv;
            if (lane < l) a0 = fma(-cl[lane], yv, a0);
            if (lane + 32 < l) a1 = fma(-cl[lane + 32], yv, a1);
          }
          if (lane < v) s_a[lane] = a0;
          if (lane + 32 < v) s_a[lane + 32] = a1;
        }
        __syncthreads();
      }
      if (v > 0) {
        // y = D^{-1} a on the columns with a valid inverse (upper triangle:
        // warps whose rows all lie below their columns skip)
        double p0 = 0.0, p1 = 0.0;
        if (g * 8 + 7 >= (row & 32)) {
#pragma unroll
          for (int q = 0; q < 8; q += 2) {
            const int j = g * 8 + q;
            if (j < v) p0 = fma(sDI[j * TB + row], s_a[j], p0);
            if (j + 1 < v) p1 = fma(sDI[(j + 1) * TB + row], s_a[j + 1], p1);
          }
        }
        sP[g * TB + row] = p0 + p1;
        __syncthreads();
        if (g == 0 && row < v) {
          const double s01 = sP[row] + sP[TB + row], s23 = sP[2 * TB + row] + sP[3 * TB + row];
          const double s45 = sP[4 * TB + row] + sP[5 * TB + row], s67 = sP[6 * TB + row] + sP[7 * TB + row];
          ycur[row] = (s01 + s23) + (s45 + s67);
        }
      }
      if (g == 0 && row < nbk) I.yP[b0 + row] = ycur[row];
      // the next block's loads go out before this block is published
      if (bi > 0) prefetch(bi - 1);
      __syncthreads();
      if (tid == 0) flag_release(yfl + bi, ep);
    }
    return true;
  }

  // Ranks >= 1: slab s (rows [SLAB s, SLAB s + SLAB), row block s / (TB/SLAB))
  // on rank 1 + s mod (size-1), largest s first.  Sums R(slab, c) y_c over
  // c = nb-1 down to row block + 2 as the blocks are published, then hands
  // the sum to rank 0.  Thread = (row, column pair); the R loads of a block
  // are issued before its flag is awaited.
  __device__ bool tri_slabs(int np, int nb, int ep) {
    constexpr int SPB = TB / SLAB;        // slabs per block
    const int nslab = SPB * (nb - 2);
    const int nh = tm.size - 1, h = tm.rank - 1;
    if (h >= nslab) return true;
    double* s_red = dyn;                  // (NT / SLAB) x SLAB
    const int row = tid & (SLAB - 1), cg = tid / SLAB;   // cg in [0, 32)
    const int* yfl = yflags();
    for (int s = h + nh * ((nslab - 1 - h) / nh); s >= 0; s -= nh) {
      const int rb = s / SPB, r0 = s * SLAB;
      double acc = 0.0;
      for (int c = nb - 1; c >= rb + 2; --c) {
        const int c0 = c * TB, nc = min(np, c0 + TB) - c0;
        const int j0 = cg, j1 = cg + 32;
        const int sl0 = (j0 < nc) ? ldcg(I.rslot + c0 + j0) : 0;
        const int sl1 = (j1 < nc) ? ldcg(I.rslot + c0 + j1) : 0;
        const double v0 = (j0 < nc) ? ldcg(Rcol(sl0) + r0 + row) : 0.0;
        const double v1 = (j1 < nc) ? ldcg(Rcol(sl1) + r0 + row) : 0.0;
        int okw = 1;
        if (tid == 0) okw = wait_ge(yfl + c, ep, tm_err(), I.wait_ns) ? 1 : 0;
        if (!__syncthreads_and(okw)) return false;
        const double y0 = (j0 < nc) ? ldcg(I.yP + c0 + j0) : 0.0;
        const double y1 = (j1 < nc) ? ldcg(I.yP + c0 + j1) : 0.0;
        acc = fma(v0, y0, acc);
        acc = fma(v1, y1, acc);
      }
      s_red[cg * SLAB + row] = acc;
      __syncthreads();
      if (warp < SLAB) {
        const double t = warp_sum(s_red[lane * SLAB + warp]);
        if (lane == 0) I.accb[r0 + warp] = t;  // read by rank 0 as its own flag
      }
      __syncthreads();
    }
    return true;
  }

  // Last ranks: inverse columns of the diagonal blocks for the positions
  // [inv_valid, np).  Item k = (block, column class mod 4) on rank
  // size-1 - k mod (size-1); one warp per column, which solves D x = e_j by
  // column-oriented substitution and writes column j of D^{-1} (zeros below
  // the diagonal).
  __device__ void tri_inverse(int np, int nb, int ep) {
    constexpr int PARTS = INV_PARTS;      // 4 column classes, one column per warp
    const int bs = inv_valid / TB;
    const int nstale = nb - bs;
    const int nitem = PARTS * nstale;
    const int nh = tm.size - 1, h = tm.size - 1 - tm.rank;
    if (nitem <= 0 || h >= nitem) return;
    double* sD = dyn;
    __shared__ double s_ri[TB];
    int* ifl = iflags();
    for (int it = h; it < nitem; it += nh) {
      // blocks in the order rank 0 needs them: nb-2, nb-3, ..., bs, and the
      // last block (which rank 0 substitutes) at the end
      const int q = it / PARTS, part = it % PARTS;
      const int bi = (q < nstale - 1) ? nb - 2 - q : nb - 1;
      const int b0 = bi * TB, nbk = min(np, b0 + TB) - b0;
      const int v = min(max(inv_valid - b0, 0), nbk);
      __syncthreads();  // the previous item's readers of sD are done
      {
        double sv[TB * TB / NT];
#pragma unroll
        for (int k = 0; k < TB * TB / NT; ++k) {
          const int idx = tid + k * NT, j = idx / TB, i = idx & (TB - 1);
          sv[k] = (j < nbk && i <= j) ? ldcg(Rcol(ldcg(I.rslot + b0 + j)) + b0 + i) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < TB * TB / NT; ++k) {
          const int idx = tid + k * NT, j = idx / TB, i = idx & (TB - 1);
          sD[j * (TB + 1) + i] = sv[k];
          if (i == j && j < nbk) s_ri[j] = rcp_nr(sv[k]);
        }
      }
      __syncthreads();
      const int j = part + PARTS * warp;
      if (j >= v && j < nbk) {
        double a0 = (lane == j) ? 1.0 : 0.0;
        double a1 = (lane + 32 == j) ? 1.0 : 0.0;
        for (int l = j; l >= 0; --l) {
          const int own = l & 31;
          const double* cl = sD + l * (TB + 1);
          double xv = (l >= 32 ? a1 : a0) * s_ri[l];
          xv = __shfl_sync(0xffffffffu, xv, own);
          if (lane == own) {
            if (l >= 32) a1 = xv; else a0 = xv;
          }
          if (lane < l) a0 = fma(-cl[lane], xv, a0);
          if (lane + 32 < l) a1 = fma(-cl[lane + 32], xv, a1);
        }
        double* out = I.Dinv + (size_t)bi * TB * TB + (size_t)j * TB;
        out[lane] = (lane <= j) ? a0 : 0.0;
        out[lane + 32] = (lane + 32 <= j) ? a1 : 0.0;
      }
      __syncthreads();
      if (tid == 0) flag_release(ifl + bi * PARTS + part, ep);
    }
  }



  // This CTA's share of the Z columns: the columns with pos < 0 that are not
  // in J[0:nj] are numbered in column order (with b = -1 appended last when
  // with_b) and split evenly over the team, so every CTA gets floor or ceil
  // of the count.  s_list receives the share in ascending order; scratch:
  // 2 ceil(n/32) words.  Returns the share's size.
  __device__ int z_share(int* s_list, unsigned* scratch, const int* s_J, int nj, bool with_b) {
    __shared__ int s_nl;
    const int nwd = (I.n + 31) >> 5;
    unsigned* s_jb = scratch;
    unsigned* s_zb = s_jb + nwd;
    for (int i = tid; i < nwd; i += NT) s_jb[i] = 0u;
    __syncthreads();
    if (tid < nj) atomicOr(&s_jb[s_J[tid] >> 5], 1u << (s_J[tid] & 31));
    __syncthreads();
    for (int w0 = warp; w0 < nwd; w0 += 4 * NW) {
      int pv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = (w0 + k * NW) * 32 + lane;
        pv[k] = (w0 + k * NW < nwd && c < I.n) ? ldcg(I.pos + c) : 0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int wd = w0 + k * NW;
        if (wd < nwd) {
          const int c = wd * 32 + lane;
          const bool z = c < I.n && pv[k] < 0 && !((s_jb[wd] >> lane) & 1u);
          const unsigned bits = __ballot_sync(0xffffffffu, z);
          if (lane == 0) s_zb[wd] = bits;
        }
      }
    }
    __syncthreads();
    if (warp == 0) {
      int nz = 0;
      for (int w0 = 0; w0 < nwd; w0 += 32) {
        int cnt = (w0 + lane < nwd) ? __popc(s_zb[w0 + lane]) : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        nz += cnt;
      }
      int lo, hi;
      split(nz + (with_b ? 1 : 0), tm.size, tm.rank, lo, hi);
      int run = 0;
      for (int w0 = 0; w0 < nwd && run < hi; w0 += 32) {
        const unsigned bits = (w0 + lane < nwd) ? s_zb[w0 + lane] : 0u;
        const int cnt = __popc(bits);
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        int r = run + inc - cnt;  // rank of this word's first Z column
        if (r < hi && r + cnt > lo) {
          unsigned bb = bits;
          while (bb) {
            const int bit = __ffs(bb) - 1;
            bb &= bb - 1;
            if (r >= lo && r < hi) s_list[r - lo] = (w0 + lane) * 32 + bit;
            ++r;
          }
        }
        run += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) {
        if (with_b && nz >= lo && nz < hi) s_list[nz - lo] = -1;
        s_nl = hi - lo;
      }
    }
    __syncthreads();
    return s_nl;
  }

  // Shared-memory layout and chunk sizes of one commit (see commit()).
  struct CommitShape {
    int L, RC1, RC2, VS;
    double* wk;        // work area
    double* s_D;       // KM x CB
    double* s_E;       // KM x CB
    const double* s_T; // packed T^T rows
    const double* s_vt;
    double* s_nrm;     // NW x CB
    const int* s_cid;  // batch columns (-1: b)
  };
  static constexpr int CB = 16;  // Z columns per commit batch

  __device__ __forceinline__ double* commit_col(const int* s_cid, int k) const {
    const int id = s_cid[k];
    return (id >= 0 ? Wcol(id) : I.bt) + nP;
  }

  // Rows [rb, rb+nr) of V (kp columns) into wk with row stride VS.
  __device__ __forceinline__ void stage_vrows(const CommitShape& cs, int rb, int nr) {
    const int tot = nr * kp;
    for (int e0 = tid; e0 < tot; e0 += 4 * NT) {
      double v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = e0 + k * NT, rr = e / kp, t = e - rr * kp, rg = rb + rr;
        v[k] = (e < tot && rg > t) ? ldcg(I.V + (size_t)rg * KM + t) : ((e < tot && rg == t) ? cs.s_vt[t] : 0.0);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = e0 + k * NT, rr = e / kp, t = e - rr * kp;
        if (e < tot) cs.wk[rr * cs.VS + t] = v[k];
      }
    }
  }

  // One batch of NB columns: D = V^T C (pass 1: thread (t1, g1) sums rows
  // g1, g1+G, ... of every chunk, then a fixed pairwise tree over g1),
  // D' = T^T D, C -= V D' and the trailing norms (pass 2: thread (r2, grp)
  // updates row r2 of every chunk in columns grp, grp+NG, ...).  NB is a
  // template parameter so that no issue slot goes to absent columns.
  template <int NB>
  __device__ void commit_batch(const CommitShape& cs) {
    const int L = cs.L, RC1 = cs.RC1, RC2 = cs.RC2, VS = cs.VS;
    double* wk = cs.wk;
    const int G = NT / kp, t1 = tid % kp, g1 = tid / kp;
    const bool act1 = g1 < G;
    double acc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = 0.0;
    double* sX = wk + RC1 * VS;  // NB x RC1
    for (int rb = 0; rb < L; rb += RC1) {
      const int nr = min(RC1, L - rb);
      __syncthreads();
      stage_vrows(cs, rb, nr);
      const int totx = NB * nr;
      for (int e0 = tid; e0 < totx; e0 += 4 * NT) {
        double v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = e0 + k * NT, cc = e / nr, rr = e - cc * nr;
          v[k] = (e < totx) ? ldcg(commit_col(cs.s_cid, cc) + rb + rr) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = e0 + k * NT, cc = e / nr, rr = e - cc * nr;
          if (e < totx) sX[cc * RC1 + rr] = v[k];
        }
      }
      __syncthreads();
      if (act1) {
        for (int rr = g1; rr < nr; rr += G) {
          const double v = wk[rr * VS + t1];
#pragma unroll
          for (int c = 0; c < NB; ++c) acc[c] = fma(v, sX[c * RC1 + rr], acc[c]);
        }
      }
    }
    __syncthreads();
    double* P = wk;  // G x kp x NB partials
    if (act1) {
#pragma unroll
      for (int c = 0; c < NB; ++c) P[(g1 * kp + t1) * NB + c] = acc[c];
    }
    __syncthreads();
    for (int st = 1; st < G; st <<= 1) {
      if (act1 && (g1 & (2 * st - 1)) == 0 && g1 + st < G) {
#pragma unroll
        for (int c = 0; c < NB; ++c) P[(g1 * kp + t1) * NB + c] += P[((g1 + st) * kp + t1) * NB + c];
      }
      __syncthreads();
    }
    for (int o = tid; o < kp * NB; o += NT) {
      const int t = o / NB, cc = o - t * NB;
      cs.s_D[t * CB + cc] = P[t * NB + cc];
    }
    __syncthreads();
    // D' = T^T D
    for (int o = tid; o < kp * NB; o += NT) {
      const int t = o % kp, cc = o / kp;
      double e2 = 0.0;
      for (int sidx = 0; sidx <= t; ++sidx) e2 = fma(cs.s_T[t * (t + 1) / 2 + sidx], cs.s_D[sidx * CB + cc], e2);
      cs.s_E[t * CB + cc] = e2;
    }
    // pass 2 (NG = 1 or 2 groups of columns)
    const int NG = NT / RC2, r2 = tid % RC2, grp = tid / RC2;
    constexpr int NK2 = (NB + 1) / 2;
    double nrm[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) nrm[k] = 0.0;
    for (int rb = 0; rb < L; rb += RC2) {
      const int nr = min(RC2, L - rb);
      __syncthreads();
      stage_vrows(cs, rb, nr);
      __syncthreads();
      if (r2 < nr) {
        const bool below = rb + r2 >= kp;
        if (NG == 1) {
          double x[NB];
#pragma unroll
          for (int k = 0; k < NB; ++k) x[k] = ldcg(commit_col(cs.s_cid, k) + rb + r2);
          for (int t = 0; t < kp; ++t) {
            const double v = wk[r2 * VS + t];
#pragma unroll
            for (int k = 0; k < NB; ++k) x[k] = fma(-v, cs.s_E[t * CB + k], x[k]);
          }
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            commit_col(cs.s_cid, k)[rb + r2] = x[k];
            if (below) nrm[k] = fma(x[k], x[k], nrm[k]);
          }
        } else {
          double x[NK2];
#pragma unroll
          for (int k = 0; k < NK2; ++k) {
            const int c = grp + 2 * k;
            x[k] = (c < NB) ? ldcg(commit_col(cs.s_cid, c) + rb + r2) : 0.0;
          }
          for (int t = 0; t < kp; ++t) {
            const double v = wk[r2 * VS + t];
#pragma unroll
            for (int k = 0; k < NK2; ++k) {
              const int c = grp + 2 * k;
              if (c < NB) x[k] = fma(-v, cs.s_E[t * CB + c], x[k]);
            }
          }
#pragma unroll
          for (int k = 0; k < NK2; ++k) {
            const int c = grp + 2 * k;
            if (c < NB) {
              commit_col(cs.s_cid, c)[rb + r2] = x[k];
              if (below) nrm[k] = fma(x[k], x[k], nrm[k]);
            }
          }
        }
      }
    }
    // norms: a group's threads are whole warps; column c = grp + NG k
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const int c = grp + NG * k;
      if (c < NB) {
        const double v = warp_sum(nrm[k]);
        if (lane == 0) cs.s_nrm[warp * CB + c] = v;
      }
    }
    __syncthreads();
    if (tid < NB) {
      const int g = tid % NG, w0 = g * (RC2 / 32);
      double v = 0.0;
      for (int w2 = 0; w2 < RC2 / 32; ++w2) v += cs.s_nrm[(w0 + w2) * CB + tid];
      if (cs.s_cid[tid] >= 0) I.u[cs.s_cid[tid]] = sqrt(v);
    }
  }

  // One batch of nb <= NBP (8 or 16) columns through the bf16 tensor cores,
  // for 5 <= kp <= 16 KT (KT = 1 or 2 tiles of 16 reflectors) with the
  // panel's reflector digits in Vd/Ver.
  //  pass 1: D = V^T C.  With V(r, :) = 2^Er v'(r, :) (|v'| < 1, digits a_k
  //    from the panel) and C' = 2^Er C (digits c_l under the column scale
  //    2^Ec), D = 2^(Ec-14) sum_lam 2^(-7 lam) sum_{k+l=lam} a_k^T c_l.
  //    64-row chunks, double-buffered: the next chunk's V digits arrive by
  //    cp.async and its C values are loaded while the tensor cores work on
  //    the current one.  Warp (tile pair, sub) takes rows sub*16 .. +15 of
  //    every chunk for one 16 x 8 (reflector, column) tile and keeps one
  //    FP32 accumulator per level k + l <= 8, moved to int32 every 128 of
  //    its rows (exact: at most 8 pairs of products below 2^14 per row).
  //  D' = T^T D in FP64.
  //  pass 2: C -= V D'.  128-row chunks, double-buffered.  From the digits
  //    of V (row scale) and of D'' = 2^Ft D' (column scale 2^Ee) warp (row
  //    tile, column tile) forms the 9 level sums of its 16 x 8 tile (exact
  //    in FP32: at most 8 pairs x 32 terms), combines them in int64
  //    (u = sum_lam lev_lam 2^(43-7 lam), levels 7 and 8 rounded down;
  //    |u| < 2^63 as lev_lam < (lam+1) 2^19) and applies x -= u 2^(Er+Ee-57)
  //    and the trailing norm in FP64.
  //  Reflector scales: V's digits are of V(r, t) / 2^Ft with 2^Ft > |v0_t|
  //    >= |V(:, t)| (the panel scales each reflector by its own power of
  //    two before the row scale is taken), so reflectors of very different
  //    norms - later columns of a correlated block keep little of their
  //    norm after the earlier reflectors - keep all their digits; the factor
  //    2^Ft returns in D (pass 1) and in D'' (pass 2).
  // Every sum is exact or in a fixed order, so the result is bitwise
  // reproducible.  Shared memory (bytes of the work area): V digit buffers
  // [0, 64K) and [64K, 128K) (R rows of 512 B: the ND digit planes side by
  // side, 16-byte chunks XOR-swizzled by row so that ldmatrix is
  // conflict-free), pass-1 C' digit buffers in the upper halves of those
  // (pass 1 has R = 64), D' digits at 128K.
  // Accuracy guard of pass 1.  The fixed-point digits carry 56 bits under
  // one power-of-two scale per V row and per column of C', so a sum whose
  // terms all lie far below the scale (a large entry of C paired with zeros
  // of V, say) loses bits that an FP64 dot product would keep.  Pass 1 also
  // forms the sum of |leading digit| products (one more MMA per step, exact
  // integers), a lower bound of sum |v'||c'| over the digit rows in units
  // of 2^(Ec - 14).  The digit result's error is at most 2L 2^(Ec-57) (times
  // 2^Ft); where that could exceed the worst-case bound of the FP64
  // evaluation, gamma_L sum |v||c| - i.e. where the digit rows' sum plus the
  // FP64 rows' sum |v||c| stays below 2^(Ec-3) (2^11 in the digits' units) -
  // the batch goes to the FP64 commit before any column is touched.
  static constexpr float GUARD1 = 2048.0f;  // 2^11: sum |v'||c'| >= 2^(Ec-3)
  static constexpr unsigned ABS2 = 0x7FFF7FFFu;  // clears the signs of a bf16 pair

  // Returns 0 when the batch is committed, 1 when a bounded wait expired, 2
  // when the accuracy guard hands the batch to the FP64 path (C untouched).
  template <int NBP, int KT>
  __device__ int commit_tc(const CommitShape& cs, int nb) {
    constexpr int NTN = NBP / 8;           // column tiles
    constexpr int COMBOS = KT * NTN;       // (reflector tile, column tile) pairs
    constexpr int MW = COMBOS * 4;         // pass-1 MMA warps
    constexpr int R1 = 64, R2 = 128;       // rows per chunk in pass 1 and 2
    constexpr int BUF = ND * 128 * 32;     // bf16 per V digit buffer
    constexpr int SB = R1 + 8;             // row stride of C' digits (bf16)
    constexpr int SE = 40;                 // row stride of D' digits (bf16)
    const int L = cs.L;
    // The digits cover rows [r0d, L); the first r0d rows - the reflectors'
    // triangle (pivots and the zeros above them, whose row scales would
    // outweigh every other row), rounded up to a multiple of 8 so that the
    // staged digit rows keep the row swizzle of Vd - are done in FP64.
    // Chunk rows below are counted from row r0d.
    const int r0d = (kp + 7) & ~7;
    const int Ld = L - r0d;
    unsigned short* sV = reinterpret_cast<unsigned short*>(cs.wk);
    unsigned short* sE = sV + 2 * BUF;
    __shared__ int s_Ec[CB], s_Ee[CB];
    const int g = lane >> 2, tq = lane & 3;
    // digit k, 16-byte chunk q (reflectors 8q .. 8q+7) of staged row r:
    // rows of 512 bytes, chunk 4k + q at (4k + q) ^ (r & 7)
    auto vaddr = [&](const unsigned short* base, int, int k, int r, int q) {
      return base + r * (16 * ND * 2) + (((4 * k + q) ^ (r & 7)) << 3);
    };
    // V digits of rows rb .. rb+R into buffer b: one bulk copy (the rows are
    // stored pre-swizzled), completing on the buffer's mbarrier; rows past L
    // are zeroed by the threads.  Every thread orders
    // its generic writes of the work area before later async copies (proxy
    // fence at entry, before pass 2 and after zeroing).
    __shared__ unsigned long long s_mbar[2];
    unsigned vph = 0u;  // bit b: parity of buffer b's next phase
    fence_proxy_async();
    if (tid == 0) {
      mbar_init(&s_mbar[0], 1);
      mbar_init(&s_mbar[1], 1);
      fence_mbar_init();
    }
    __syncthreads();
    auto stage_v = [&](int rb, int R, int b) {
      unsigned short* dst = sV + b * BUF;
      const int nr = min(R, Ld - rb);
      if (tid == 0) {
        mbar_expect_tx(&s_mbar[b], (unsigned)(nr * 64 * ND));
        bulk_g2s(dst, I.Vd + (size_t)(r0d + rb) * (16 * ND), (unsigned)(nr * 64 * ND), &s_mbar[b]);
      }
      if (nr < R) {
        for (int e = nr * 4 * ND + tid; e < R * 4 * ND; e += NT)
          *reinterpret_cast<uint4*>(dst + e * 8) = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async();
      }
    };
    // wait for buffer b's copies (bounded); false on expiry
    auto wait_v = [&](int b) -> bool {
      const unsigned par = (vph >> b) & 1u;
      vph ^= 1u << b;
      const long long t0 = gtimer();
      unsigned spins = 0;
      while (!mbar_try_wait(&s_mbar[b], par)) {
        if ((++spins & 255u) == 0u && gtimer() - t0 > WAIT_NS) return false;
      }
      return true;
    };
    auto expired = [&]() {
      if (tid == 0) {
        int* er = tm_err();
        if (er) atomicExch(er, 1);
      }
    };
    // column scales of C' = 2^Er C: (column, row quarter) per warp, 8 rows
    // per lane in flight
    if (tid < CB) s_Ec[tid] = -8000;
    __syncthreads();
    for (int p = warp; p < nb * 4; p += NW) {
      const int c = p >> 2;
      const double* col = commit_col(cs.s_cid, c) + r0d;
      const int* ver = I.Ver + r0d;
      int lo, hi;
      split(Ld, 4, p & 3, lo, hi);
      int mx = -8000;
      for (int r0 = lo + lane; r0 < hi; r0 += 256) {
        double xv[8];
        int ev[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int r = r0 + 32 * u;
          xv[u] = (r < hi) ? ldcg(col + r) : 0.0;
          ev[u] = (r < hi) ? ldcg(ver + r) : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = ebound(xv[u]);
          if (e > -2000) mx = max(mx, e + ev[u]);
        }
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) atomicMax(&s_Ec[c], mx);
    }
    __syncthreads();
    // ---- pass 1
    const int nch1 = (Ld + R1 - 1) / R1;
    const bool mw = warp < MW;
    const int cmb = warp % COMBOS, sub = warp / COMBOS;
    const int mt = cmb % KT, nt = cmb / KT;
    // C' digits: thread (column tid/32, row pair tid%32) of each chunk, from
    // the chunk's C values and row exponents, staged by cp.async in the
    // buffer's [50K, 58.25K) bytes
    const bool dw = tid < NBP * 32;
    const int dc = tid >> 5, drr = 2 * (tid & 31);
    const int dec = (dw && dc < nb) ? s_Ec[dc] : 0;
    auto cstage = [&](int b) { return reinterpret_cast<double*>(sV + b * BUF) + 6400; };
    auto stage_c = [&](int rb, int b) {
      double* sC = cstage(b);
      int* sR = reinterpret_cast<int*>(sC + NBP * R1);
      for (int e = tid; e < NBP * R1; e += NT) {
        const int c = e / R1, r = e - c * R1;
        const bool ok = c < nb && rb + r < Ld;
        cp8(sC + e, ok ? commit_col(cs.s_cid, c) + r0d + rb + r : I.u, ok);
      }
      if (tid < R1) cp4(sR + tid, rb + tid < Ld ? I.Ver + r0d + rb + tid : I.Ver, rb + tid < Ld);
      cp_commit();
    };
    auto digits_c = [&](int b) {
      if (!dw) return;
      const double* sC = cstage(b);
      const int* sR = reinterpret_cast<const int*>(sC + NBP * R1);
      const double xa = sC[dc * R1 + drr], xb = sC[dc * R1 + drr + 1];
      unsigned short* sBb = sV + b * BUF + BUF / 2;
      unsigned ha, la, hb, lb, sg, nb2;
      halves28(fix56(xa, sR[drr] + 56 - dec), ha, la);
      halves28(fix56(xb, sR[drr + 1] + 56 - dec), hb, lb);
      sign2(xa < 0.0, xb < 0.0, sg, nb2);
#pragma unroll
      for (int k = 0; k < ND; ++k) *reinterpret_cast<unsigned*>(sBb + (k * NBP + dc) * SB + drr) = dig2k(k, ha, la, hb, lb, sg, nb2);
    };
    // levels 0 .. NEX-1 move every 128 rows into exact int32 sums in shared
    // memory (shared atomics: exact, so the order of the warps does not
    // matter); levels NEX .. 8 stay in FP32, where their rounding weighs
    // below 2^-54 of the scales
    constexpr int NEX = 7;
    int* sF = reinterpret_cast<int*>(reinterpret_cast<char*>(sV) + 131072);  // COMBOS x NEX x 32 x 4
    for (int e = tid; e < COMBOS * NEX * 128; e += NT) sF[e] = 0;
    float acc[NLV][4];
#pragma unroll
    for (int l = 0; l < NLV; ++l)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[l][j] = 0.f;
    float gacc[4] = {0.f, 0.f, 0.f, 0.f};  // sum of |leading digit| products (guard)
    int since = 0;
    // every CTA walks the chunks from its own starting chunk, so that the
    // CTAs do not all ask for the same digit rows at the same moment (the
    // sums are exact, so the order does not matter)
    const int s1 = tm.rank % nch1;
    auto row1 = [&](int jc) { return ((jc + s1) % nch1) * R1; };
    stage_c(row1(0), 0);
    stage_v(row1(0), R1, 0);
    cp_wait_all();
    __syncthreads();
    digits_c(0);
    for (int jc = 0; jc < nch1; ++jc) {
      const int b = jc & 1;
      const bool okv = wait_v(b);
      if (__syncthreads_or(!okv)) {
        expired();
        return 1;
      }
      if (jc + 1 < nch1) {
        stage_c(row1(jc + 1), b ^ 1);
        stage_v(row1(jc + 1), R1, b ^ 1);
      }
      if (mw) {
        const unsigned short* sAb = sV + b * BUF;
        const unsigned short* sBb = sAb + BUF / 2;
        const int r0 = sub * 16;
        unsigned bq[ND][2];
#pragma unroll
        for (int l = 0; l < ND; ++l) ldsm_x2(bq[l], sBb + (l * NBP + nt * 8 + (lane & 7)) * SB + r0 + ((lane >> 3) & 1) * 8);
        const int ra = r0 + (lane & 7) + ((lane >> 4) << 3), qa = mt * 2 + ((lane >> 3) & 1);
#pragma unroll
        for (int k = 0; k < ND; ++k) {
          unsigned a[4];
          ldsm_x4_t(a, vaddr(sAb, R1, k, ra, qa));
#pragma unroll
          for (int l = 0; l < ND && k + l < NLV; ++l) mma_bf16(acc[k + l], a, bq[l]);
          if (k == 0) {
            const unsigned ga[4] = {a[0] & ABS2, a[1] & ABS2, a[2] & ABS2, a[3] & ABS2};
            const unsigned gb[2] = {bq[0][0] & ABS2, bq[0][1] & ABS2};
            mma_bf16(gacc, ga, gb);
          }
        }
      }
      if (jc + 1 < nch1) {
        cp_wait_all();  // the next chunk's C values (its V digits may still be in flight)
        __syncthreads();
        digits_c(b ^ 1);
      }
      since += 16;
      if (mw && (since == 128 || jc + 1 == nch1)) {
#pragma unroll
        for (int l = 0; l < NEX; ++l)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            atomicAdd(sF + ((cmb * NEX + l) * 32 + lane) * 4 + j, __float2int_rn(acc[l][j]));
            acc[l][j] = 0.f;
          }
      }
      if (since == 128) since = 0;
    }
    // levels NEX .. 8 summed over the sub-blocks in order, then D from the
    // level sums
    __syncthreads();
    constexpr int NST = NLV - NEX + 1;  // staged FP32 sums per warp: levels NEX .. 8 and the guard
    float* sStage = reinterpret_cast<float*>(sV);                                 // MW x NST x 32 x 4
    double* sL = reinterpret_cast<double*>(reinterpret_cast<char*>(sV) + 73728);  // NLV x 32 x NBP
    __shared__ int s_guard;
    if (tid == 0) s_guard = 0;
    if (mw) {
#pragma unroll
      for (int l = NEX; l < NLV; ++l)
#pragma unroll
        for (int j = 0; j < 4; ++j) sStage[((warp * NST + l - NEX) * 32 + lane) * 4 + j] = acc[l][j];
#pragma unroll
      for (int j = 0; j < 4; ++j) sStage[((warp * NST + NST - 1) * 32 + lane) * 4 + j] = gacc[j];
    }
    __syncthreads();
    // the guard's sums of |leading digit| products per (reflector, column),
    // added over the four row sub-blocks (checked with D below)
    float* sG = reinterpret_cast<float*>(reinterpret_cast<char*>(sV) + 32768);  // KM x CB
    for (int e = tid; e < COMBOS * 128; e += NT) {
      const int j = e & 3, ln = (e >> 2) & 31, cb = e >> 7;
      const int t = (cb % KT) * 16 + (ln >> 2) + ((j >> 1) << 3), c = (cb / KT) * 8 + 2 * (ln & 3) + (j & 1);
      if (t < kp && c < nb) {
        float g = 0.f;
        for (int sb = 0; sb < 4; ++sb) g += sStage[(((sb * COMBOS + cb) * NST + NST - 1) * 32 + ln) * 4 + j];
        sG[t * CB + c] = g;
      }
    }
    for (int e = tid; e < COMBOS * NLV * 128; e += NT) {
      const int j = e & 3, ln = (e >> 2) & 31, lam = (e >> 7) % NLV, cb = (e >> 7) / NLV;
      double v = 0.0;
      if (lam < NEX) {
        v = (double)sF[((cb * NEX + lam) * 32 + ln) * 4 + j];
      } else {
        for (int sb = 0; sb < 4; ++sb)
          v += (double)sStage[(((sb * COMBOS + cb) * NST + lam - NEX) * 32 + ln) * 4 + j];
      }
      const int t = (cb % KT) * 16 + (ln >> 2) + ((j >> 1) << 3), c = (cb / KT) * 8 + 2 * (ln & 3) + (j & 1);
      sL[(lam * 32 + t) * NBP + c] = v;
    }
    __syncthreads();
    for (int o = tid; o < kp * nb; o += NT) {
      const int t = o / nb, c = o - t * nb;
      double s = sL[((NLV - 1) * 32 + t) * NBP + c];
      for (int lam = NLV - 2; lam >= 0; --lam) s = fma(s, 0x1p-7, sL[(lam * 32 + t) * NBP + c]);
      // rows t .. r0d-1 in FP64 (V(r, t) = 0 above row t), with sum |v||c|
      const double* col = commit_col(cs.s_cid, c);
      double tri = 0.0, tabs = 0.0;
      for (int r = t; r < r0d; ++r) {
        const double vr = (r > t) ? ldcg(I.V + (size_t)r * KM + t) : cs.s_vt[t], cr = ldcg(col + r);
        tri = fma(vr, cr, tri);
        tabs = fma(fabs(vr), fabs(cr), tabs);
      }
      const int es = s_Ec[c] + ebound(cs.s_vt[t]);  // 2^Ft: the reflector's scale
      cs.s_D[t * CB + c] = ldexp(s, es - 14) + tri;
      // guard: the digits' error (at most 2L 2^(es-57)) must stay within
      // gamma_L sum |v||c|, whose lower bound is 2^(es-14) sG + tabs; a
      // column without digit rows (all zero below r0d) has no digit error
      if (s_Ec[c] > -8000 && !(ldexp((double)sG[t * CB + c], es - 14) + tabs >= ldexp((double)GUARD1, es - 14)))
        s_guard = 1;
    }
    __syncthreads();
    // bf16 MMAs of pass 1: per chunk, each MMA warp's 16 rows take the 43
    // digit pairs and the guard's
    const double mma1 = (double)MW * nch1 * 44.0;
    if (s_guard || I.guard_force == 1) {
      if (tid == 0) {
        atomicAdd(I.ctl + C_GUARD1, 1);
        if (I.phase_ns) atomicAdd(I.phase_ns + 2 * NPHASE, mma1);
      }
      return 2;
    }
    // D' = T^T D
    for (int o = tid; o < kp * nb; o += NT) {
      const int t = o % kp, cc = o / kp;
      double e2 = 0.0;
      for (int sidx = 0; sidx <= t; ++sidx) e2 = fma(cs.s_T[t * (t + 1) / 2 + sidx], cs.s_D[sidx * CB + cc], e2);
      cs.s_E[t * CB + cc] = e2;
    }
    __syncthreads();
    // digits of D' under a column scale: warp c, lane t
    for (int c = warp; c < NBP; c += NW) {
      const double v = (c < nb && lane < kp) ? scale2(cs.s_E[lane * CB + c], ebound(cs.s_vt[lane])) : 0.0;
      const int ee = __reduce_max_sync(0xffffffffu, ebound(v));
      unsigned ha, la;
      halves28(fix56(v, 56 - ee), ha, la);
      const unsigned hb = __shfl_down_sync(0xffffffffu, ha, 1), lb = __shfl_down_sync(0xffffffffu, la, 1);
      const bool nega = v < 0.0;
      const bool negb = __shfl_down_sync(0xffffffffu, nega ? 1 : 0, 1) != 0;
      unsigned sg, nb2;
      sign2(nega, negb, sg, nb2);
      if ((lane & 1) == 0) {
#pragma unroll
        for (int k = 0; k < ND; ++k) *reinterpret_cast<unsigned*>(sE + (k * NBP + c) * SE + lane) = dig2k(k, ha, la, hb, lb, sg, nb2);
      }
      if (lane == 0) s_Ee[c] = ee;
    }
    __syncthreads();
    // ---- pass 2 (digit rows r0d .. L-1; rows below r0d after the loop)
    const int nch2 = (Ld + R2 - 1) / R2;
    const bool act2 = warp < 8 * NTN;
    const int rt = warp & 7, nt2 = warp >> 3;
    const int c0 = nt2 * 8 + 2 * tq;
    double nrm0 = 0.0, nrm1 = 0.0;
    const int s2 = tm.rank % nch2;
    auto row2 = [&](int jc) { return ((jc + s2) % nch2) * R2; };
    fence_proxy_async();  // pass-1 scratch writes before the async copies
    __syncthreads();
    stage_v(row2(0), R2, 0);
    for (int jc = 0; jc < nch2; ++jc) {
      const int rb = row2(jc), b = jc & 1;
      const bool okv = wait_v(b);
      if (__syncthreads_or(!okv)) {
        expired();
        return 1;
      }
      if (jc + 1 < nch2) stage_v(row2(jc + 1), R2, b ^ 1);
      if (act2) {
        // this thread's four elements: rows ra, ra + 8; columns c0, c0 + 1
        const int ra = r0d + rb + rt * 16 + g, rb8 = ra + 8;
        double xv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = c0 + (j & 1), row = (j < 2) ? ra : rb8;
          xv[j] = (act2 && c < nb && row < L) ? ldcg(commit_col(cs.s_cid, c) + row) : 0.0;
        }
        const int er0 = (ra < L) ? ldcg(I.Ver + ra) : 0, er1 = (rb8 < L) ? ldcg(I.Ver + rb8) : 0;
        float a2[NLV][4];
#pragma unroll
        for (int l = 0; l < NLV; ++l)
#pragma unroll
          for (int j = 0; j < 4; ++j) a2[l][j] = 0.f;
        const unsigned short* sAb = sV + b * BUF;
        const int r0 = rt * 16, rq = r0 + (lane & 7) + ((lane >> 3) & 1) * 8;
#pragma unroll
        for (int ks = 0; ks < KT; ++ks) {
          unsigned eb[ND][2];
#pragma unroll
          for (int l = 0; l < ND; ++l)
            ldsm_x2(eb[l], sE + (l * NBP + nt2 * 8 + (lane & 7)) * SE + ks * 16 + ((lane >> 3) & 1) * 8);
#pragma unroll
          for (int k = 0; k < ND; ++k) {
            unsigned a[4];
            ldsm_x4(a, vaddr(sAb, R2, k, rq, ks * 2 + ((lane >> 4) & 1)));
#pragma unroll
            for (int l = 0; l < ND && k + l < NLV; ++l) mma_bf16(a2[k + l], a, eb[l]);
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int row = (j < 2) ? ra : rb8;
          const int c = c0 + (j & 1);
          if (c < nb && row < L) {
            double* p = commit_col(cs.s_cid, c);
            long long u = 0;
#pragma unroll
            for (int l = 0; l < 7; ++l) u += (long long)__float2int_rn(a2[l][j]) * (1ll << (43 - 7 * l));
            u += (long long)(__float2int_rn(a2[7][j]) >> 6);
            u += (long long)(__float2int_rn(a2[8][j]) >> 13);
            const int es = max(-2044, ((j < 2) ? er0 : er1) + s_Ee[c] - 57);
            const double x = xv[j] - ll_scaled(u, es);
            p[row] = x;
            if (row >= kp) {
              if (j & 1) nrm1 = fma(x, x, nrm1);
              else nrm0 = fma(x, x, nrm0);
            }
          }
        }
      }
    }
    // rows r < r0d in FP64, in the order of the FP64 commit; rows kp .. r0d-1
    // belong to the trailing norm: kept for a fixed-order sum per column (in
    // rows 8 .. 15 of s_nrm, which the row tiles below leave free)
    double* s_tx = cs.s_nrm + 8 * CB;
    for (int o = tid; o < r0d * nb; o += NT) {
      const int r = o / nb, c = o - r * nb;
      double* col = commit_col(cs.s_cid, c);
      double x = ldcg(col + r);
      for (int t = 0; t <= min(r, kp - 1); ++t)
        x = fma(-((r > t) ? ldcg(I.V + (size_t)r * KM + t) : cs.s_vt[t]), cs.s_E[t * CB + c], x);
      col[r] = x;
      if (r >= kp) s_tx[(r - kp) * CB + c] = x;
    }
    // trailing norms: lanes of one column quad, then the 8 row tiles in order
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      nrm0 += __shfl_xor_sync(0xffffffffu, nrm0, o);
      nrm1 += __shfl_xor_sync(0xffffffffu, nrm1, o);
    }
    if (act2 && lane < 4) {
      cs.s_nrm[rt * CB + nt2 * 8 + 2 * lane] = nrm0;
      cs.s_nrm[rt * CB + nt2 * 8 + 2 * lane + 1] = nrm1;
    }
    __syncthreads();
    if (tid < nb) {
      double v = 0.0;
      for (int r8 = 0; r8 < 8; ++r8) v += cs.s_nrm[r8 * CB + tid];
      for (int r = kp; r < r0d; ++r) v = fma(s_tx[(r - kp) * CB + tid], s_tx[(r - kp) * CB + tid], v);
      if (cs.s_cid[tid] >= 0) I.u[cs.s_cid[tid]] = sqrt(v);
    }
    if (tid == 0 && I.phase_ns)  // pass 2: 43 digit pairs per 16 x 8 tile and 16 reflectors
      atomicAdd(I.phase_ns + 2 * NPHASE, mma1 + (double)(8 * NTN) * nch2 * KT * 43.0);
    return 0;
  }


  // Commit for kp <= 4 (one-column LH steps and short J): V staged once for
  // all L rows, then one warp per column does D = V^T x (lanes over rows,
  // fixed-order sums), D' = T^T D, x -= V D' and the trailing norm, with no
  // CTA-wide reduction.  The sums depend on kp alone.
  template <int KP>
  __device__ void commit_small(int L, double* sV, const int* s_list, int nl) {
    for (int e0 = tid; e0 < L * KP; e0 += 8 * NT) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int e = e0 + j * NT, r = e / KP, t = e - r * KP;
        v[j] = (e < L * KP && r > t) ? ldcg(I.V + (size_t)r * KM + t)
                                     : ((e < L * KP && r == t) ? ldcg(I.vtop + t) : 0.0);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (e0 + j * NT < L * KP) sV[e0 + j * NT] = v[j];
    }
    double Tm[KP][KP];
#pragma unroll
    for (int a = 0; a < KP; ++a)
#pragma unroll
      for (int c = 0; c < KP; ++c) Tm[a][c] = (a <= c) ? ldcg(I.T + a + c * KM) : 0.0;
    __syncthreads();
    for (int k = warp; k < nl; k += NW) {
      const int id = s_list[k];
      double* x = (id >= 0 ? Wcol(id) : I.bt) + nP;
      // eight rows per lane in flight in both passes
      double acc[KP][2];
#pragma unroll
      for (int t = 0; t < KP; ++t) acc[t][0] = acc[t][1] = 0.0;
      int r = lane;
      for (; r + 224 < L; r += 256) {
        double xv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) xv[j] = ldcg(x + r + 32 * j);
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int t = 0; t < KP; ++t) acc[t][j & 1] = fma(sV[(r + 32 * j) * KP + t], xv[j], acc[t][j & 1]);
      }
      for (; r < L; r += 32) {
        const double xv = ldcg(x + r);
#pragma unroll
        for (int t = 0; t < KP; ++t) acc[t][0] = fma(sV[r * KP + t], xv, acc[t][0]);
      }
      double D[KP], E[KP];
#pragma unroll
      for (int t = 0; t < KP; ++t) D[t] = warp_sum(acc[t][0] + acc[t][1]);
#pragma unroll
      for (int t = 0; t < KP; ++t) {
        double e2 = 0.0;
#pragma unroll
        for (int a = 0; a <= t; ++a) e2 = fma(Tm[a][t], D[a], e2);
        E[t] = e2;
      }
      double nrm0 = 0.0, nrm1 = 0.0;
      for (int r0 = 0; r0 < L; r0 += 256) {
        double xv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int rr = r0 + lane + 32 * j;
          xv[j] = (rr < L) ? ldcg(x + rr) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int rr = r0 + lane + 32 * j;
          if (rr < L) {
            double v = xv[j];
#pragma unroll
            for (int t = 0; t < KP; ++t) v = fma(-sV[rr * KP + t], E[t], v);
            x[rr] = v;
            if (rr >= KP) {
              if (j & 1) nrm1 = fma(v, v, nrm1);
              else nrm0 = fma(v, v, nrm0);
            }
          }
        }
      }
      const double nrm = warp_sum(nrm0 + nrm1);
      if (lane == 0 && id >= 0) I.u[id] = sqrt(nrm);
    }
  }

  // ------------------------------------------------------------ commit
  // Makes J[0:kp] passive: new R columns [W(0:nP, J); R22], the block
  // reflector I - V T^T V^T applied to the trailing rows of every Z column
  // and of Q^T b, and u = ||C|| for the Z columns (Algorithm 3, rank-k update
  // and column norms of C).
  __device__ __forceinline__ bool commit(const int* s_J) {
    const int L = I.m - nP;
    flops(PH_COMMIT, 4.0 * kp * (double)L * (double)(I.n - nP - kp + 1) + 2.0 * (double)L * (I.n - nP - kp));
    // (a) R columns of the new positions (free slots rslot[nP..nP+kp))
    {
      const int gt = tm.rank * NT + tid, nt = tm.size * NT;
      const int tot = (nP + KM) * kp;
      for (int e = gt; e < tot; e += nt) {
        const int t = e / (nP + KM), row = e - t * (nP + KM);
        const int slot = ldcg(I.rslot + nP + t);
        if (row < nP) Rcol(slot)[row] = ldcg(Wcol(s_J[t]) + row);
        else if (row - nP <= t) Rcol(slot)[row] = ldcg(I.R22 + (row - nP) + t * KM);
      }
      if (tm.rank == 0 && tid < kp) {
        I.order[nP + tid] = s_J[tid];
        I.pos[s_J[tid]] = nP + tid;
        I.xP[nP + tid] = 0.0;
        I.yP[nP + tid] = ldcg(I.yJ + tid);
        if (sgn) I.csign[s_J[tid]] = ldcg(I.w + s_J[tid]) < 0.0 ? -1 : 1;
      }
    }
    // (b) trailing update of the Z columns and of Q^T b: D = V^T C (pass 1),
    // D' = T^T D, C -= V D' and the new trailing norms (pass 2).  The Z
    // columns are numbered in column order (b last) and split evenly over
    // the team, in batches of CB columns per CTA.  V's triangular structure
    // (zero above row t, v0 on row t) is folded into the staged rows.  Every
    // sum runs in an order fixed by kp alone.
    if (kp <= 0) {
      nP += kp;
      return sync();
    }
    const int VS = kp | 1;                          // odd row stride of staged V rows
    double* s_D = dyn;                              // KM x CB
    double* s_E = dyn + KM * CB;                    // KM x CB
    double* wk = dyn + 2 * KM * CB;                 // work area
    constexpr int WKD = DYN_SMEM / 8 - 2 * KM * CB; // its size in doubles
    const int RC1 = min(1024, (WKD / (VS + CB)) & ~31);  // pass-1 rows per chunk
    const int RC2 = (WKD / VS >= 512) ? 512 : (WKD / VS >= 256) ? 256 : (WKD / VS >= 128) ? 128 : 64;
    __shared__ double s_T[KM * KM / 2 + KM];
    __shared__ double s_vt[KM];
    __shared__ double s_nrm[NW * CB];
    __shared__ int s_cid[CB];
    __shared__ int s_list[CAND_LOCAL_MAX + 1];
    for (int e = tid; e < kp * kp; e += NT) {
      const int t = e / kp, sidx = e - t * kp;
      if (sidx <= t) s_T[t * (t + 1) / 2 + sidx] = ldcg(I.T + sidx + t * KM);
    }
    if (tid < kp) s_vt[tid] = ldcg(I.vtop + tid);
    const int nl_share = z_share(s_list, reinterpret_cast<unsigned*>(wk), s_J, kp, true);
    const int nl = nl_share;
    if (kp <= 4 && L * kp <= WKD) {
      __syncthreads();  // z_share's scratch in wk is free again
      switch (kp) {
        case 1: commit_small<1>(L, wk, s_list, nl); break;
        case 2: commit_small<2>(L, wk, s_list, nl); break;
        case 3: commit_small<3>(L, wk, s_list, nl); break;
        default: commit_small<4>(L, wk, s_list, nl); break;
      }
      nP += kp;
      return sync();
    }
    const CommitShape cs{L, RC1, RC2, VS, wk, s_D, s_E, s_T, s_vt, s_nrm, s_cid};
    // the tensor-core form needs this panel's reflector digits
    const bool tc = vd_ok && kp > 4 && kp <= 32 && L <= 16384 && L >= kp + 72;  // int32 level sums
    for (int base = 0; base < nl; base += CB) {
      const int nb = min(CB, nl - base);
      __syncthreads();
      if (tid < nb) s_cid[tid] = s_list[base + tid];
      __syncthreads();
      if (tc) {
        int r;
        if (kp <= 16) r = (nb <= 8) ? commit_tc<8, 1>(cs, nb) : commit_tc<16, 1>(cs, nb);
        else r = (nb <= 8) ? commit_tc<8, 2>(cs, nb) : commit_tc<16, 2>(cs, nb);
        if (r == 1) return false;
        if (r == 0) continue;
        __syncthreads();  // r == 2: the FP64 commit below takes this batch
      }
      switch (nb) {
        case 1: commit_batch<1>(cs); break;
        case 2: commit_batch<2>(cs); break;
        case 3: commit_batch<3>(cs); break;
        case 4: commit_batch<4>(cs); break;
        case 5: commit_batch<5>(cs); break;
        case 6: commit_batch<6>(cs); break;
        case 7: commit_batch<7>(cs); break;
        case 8: commit_batch<8>(cs); break;
        case 9: commit_batch<9>(cs); break;
        case 10: commit_batch<10>(cs); break;
        case 11: commit_batch<11>(cs); break;
        case 12: commit_batch<12>(cs); break;
        case 13: commit_batch<13>(cs); break;
        case 14: commit_batch<14>(cs); break;
        case 15: commit_batch<15>(cs); break;
        default: commit_batch<16>(cs); break;
      }
    }
    nP += kp;
    return sync();
  }

  // ------------------------------------------------------------ inner loop
  // Algorithm 3 inner loop: step length alpha, x update, removal set Q,
  // Givens downdate (Algorithm 5, one deleted position at a time from the
  // highest), re-solve.
  __device__ bool inner_loop() {
    __shared__ double shv[32];
    __shared__ int shi[32];
    int steps = 0;
    if (sgn == 2) {
      // sign flip (section 4.2): a passive column whose y in [A -A] is
      // negative gives way to its twin, whose R column is the negated one,
      // so the physical R, y and W stay as they are and only the sign
      // changes; the twin was in Z, so its previous iterate is 0.  Exact
      // zeros of y are left to the ordinary inner step below.
      __shared__ int s_nf;
      if (tm.rank == 0) {
        int nf = 0;
        for (int p = tid; p < nP; p += NT) {
          const int c = ldcg(I.order + p);
          const int sc = ldcg(I.csign + c);
          if ((double)sc * ldcg(I.yP + p) < 0.0) {
            I.csign[c] = -sc;
            I.xP[p] = 0.0;
            ++nf;
          }
        }
        nf = block_sum_int(nf, shi);
        if (tid == 0) I.ctl[C_NFLIP] = nf;
      }
      if (!sync()) return false;
      if (tid == 0) s_nf = ldcg(I.ctl + C_NFLIP);
      __syncthreads();
      n_flip += s_nf;
    }
    for (;;) {
      // any y_P <= 0 ?  (with the positivity trick: y of the signed column)
      int neg = 0;
      for (int p = tid; p < nP; p += NT) neg |= (pos_sign(p) * ldcg(I.yP + p) <= 0.0);
      neg = block_sum_int(neg, shi);
      if (!neg) return true;
      if (steps > nP + 1) {
        status = LHDM_ERR_MAX_ITER;
        return true;
      }
      ++steps;
      ++n_inner;
      // alpha = min x_p/(x_p - y_p) over y_p <= 0; i* lowest column on ties
      ArgMax best{0.0, -1};
      for (int p = tid; p < nP; p += NT) {
        const double yp = ldcg(I.yP + p), sg = pos_sign(p);
        if (sg * yp <= 0.0) {
          // x/(x - y) is the same for the signed column (signs cancel)
          const double xp = ldcg(I.xP + p);
          const double t = xp / (xp - yp);
          const int c = ldcg(I.order + p);
          // minimise t: use (-t, c) in the argmax with lowest-index ties
          // (the index in [A -A] with the positivity trick)
          best = amax_merge(best, ArgMax{-t, sg < 0.0 ? c + I.n : c});
        }
      }
      best = block_amax(best, shv, shi);
      const double alpha = -best.v;
      const int istar = best.i;
      // x update and removal set (rank 0 writes; positions listed descending)
      __shared__ int s_nq;
      int* qlist = I.qlist;
      if (tm.rank == 0) {
        if (tid == 0) s_nq = 0;
        __syncthreads();
        for (int p = tid; p < nP; p += NT) {
          const double xp = ldcg(I.xP + p), yp = ldcg(I.yP + p), sg = pos_sign(p);
          double xn = xp + alpha * (yp - xp);
          const int c = ldcg(I.order + p);
          if ((sg < 0.0 ? c + I.n : c) == istar) xn = 0.0;
          if (sg * xn <= 0.0) {
            xn = 0.0;
            const int k = atomicAdd(&s_nq, 1);
            qlist[k] = p;
          }
          I.xP[p] = xn;
        }
        __syncthreads();
        if (tid == 0) {
          // sort descending (few entries)
          const int nq = s_nq;
          for (int a = 1; a < nq; ++a) {
            const int v = qlist[a];
            int bb = a - 1;
            while (bb >= 0 && qlist[bb] < v) { qlist[bb + 1] = qlist[bb]; --bb; }
            qlist[bb + 1] = v;
          }
          I.ctl[C_NRUN] = nq;
        }
      }
      if (!sync()) return false;
      const int nq = ldcg(I.ctl + C_NRUN);
      removed += nq;
      ++inner_step;
      for (int k = 0; k < nq; ++k) {
        const int q = ldcg(I.qlist + k);
        if (!delete_position(q)) return false;
      }
      // re-solve: rhs = (Q^T b)[0:nP] was written by the owner of b
      phase(PH_ITRSV);
      if (!trsv(nP)) return false;
      phase(PH_INNER);
    }
  }


  // Deletes position q of R (Algorithm 5 for one column): bookkeeping, the
  // rotation chain over positions q..nP-2 generated in blocks of DB
  // positions (block b on CTA b mod size, handed over through a published
  // counter), then the same rotations applied to every Z column and to b.
  __device__ bool delete_position(int q) {
    const int np = nP;
    inv_valid = min(inv_valid, q);
    const int nrot = np - 1 - q;
    flops(PH_CHAIN, 3.0 * (double)nrot * (nrot + 1));
    flops(PH_ZROT, 6.0 * (double)nrot * (double)(I.n - np + 2));
    if (tm.rank == 0) {
      // the removed column re-enters Z in trailing form: W(:, c) = [R(0:q, slot); 0]
      const int c = ldcg(I.order + q);
      const int sq = ldcg(I.rslot + q);
      double* wc = Wcol(c);
      for (int i = tid; i < I.m; i += NT) wc[i] = (i <= q) ? ldcg(Rcol(sq) + i) : 0.0;
      // its trailing norm is built up below like every Z column's
      if (tid == 0) I.u[c] = 0.0;
      // shift positions q+1..np-1 down by one (read all, then write all)
      const int cnt = np - 1 - q;
      constexpr int PER = 8;  // positions per thread per sweep
      for (int base = 0; base < cnt; base += NT * PER) {
        int oc[PER], sl[PER];
        double xv[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int p = q + base + tid + k * NT;
          oc[k] = (p < np - 1) ? ldcg(I.order + p + 1) : -1;
          sl[k] = (p < np - 1) ? ldcg(I.rslot + p + 1) : 0;
          xv[k] = (p < np - 1) ? ldcg(I.xP + p + 1) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const int p = q + base + tid + k * NT;
          if (p < np - 1) {
            I.order[p] = oc[k];
            I.rslot[p] = sl[k];
            I.xP[p] = xv[k];
            I.pos[oc[k]] = p;
          }
        }
        __syncthreads();
      }
      if (tid == 0) {
        I.pos[c] = -1;
        I.rslot[np - 1] = sq;
        I.order[np - 1] = -1;
        I.xP[np - 1] = 0.0;
      }
    }
    // the rotation log starts empty: every slot holds NaN until its value is
    // published (each slot is written once, so a reader needs no fence)
    for (int i = tm.rank * NT + tid; i < nrot; i += tm.size * NT) {
      I.rotc[i] = __longlong_as_double(0x7ff8000000000000LL);
      I.rots[i] = __longlong_as_double(0x7ff8000000000000LL);
    }
    if (!sync()) return false;
    phase(PH_CHAIN);
    // (i) rotation chain: the rotations only (R's rotated rows are written
    // with the Z columns in (ii)).  Block b covers generating positions
    // [q + b*DB, q + (b+1)*DB) on CTA b mod size; lane l of warp 0 owns
    // position bs + l.  Warp 0 first carries its columns' running row value
    // through the earlier blocks' rotations as they appear in the log, then
    // generates the block's rotations; warp 2 forms their scales, warp 1
    // turns them into cosines and sines and publishes them.  Each warp issues one FP64 instruction per
    // 64 cycles on its SM sub-partition, so the per-rotation FP64 work on
    // the dependent chain is kept to two instructions.
    const int nblk = (nrot + DB - 1) / DB;
    // the ranks the chain leaves free apply the rotations as they appear
    // (when they are at least a quarter of the team and the log fits one
    // shared-memory stage); otherwise every rank applies them afterwards
    bool follow = false;
    if constexpr (std::is_same<Team, GridTeam>::value)
      follow = nrot > 0 && nrot <= ROT_STAGE && 4 * (tm.size - nblk) >= tm.size;
    double* sB = dyn;                  // sB[e][l] = R(bs+1+e, position bs+l), DB x (DB+1)
    double* sY = dyn + DB * (DB + 1);  // -sB[e][l] / sB[e][e] (the one-FMA form below)
    __shared__ double s_ra[DB], s_rq[DB], s_rqa[DB];
    __shared__ int s_rk[DB], s_rid[DB];
    __shared__ int s_prog, s_qprog;  // rotations generated / with their scale (-1: abandoned)
    volatile int* prog = &s_prog;
    volatile int* qprog = &s_qprog;
    // A one-CTA team runs the blocks one after another, so it keeps every
    // later position's running row value in shared memory and carries all
    // of them through each block's rotations as soon as they are out, with
    // every thread (one FP64 pipe per sub-partition) instead of the next
    // block's warp 0 replaying the whole log on one.
    double* s_car = dyn + 2 * DB * (DB + 1);
    __shared__ double s_rc[DB], s_rs[DB];
    bool car = false;
    if constexpr (std::is_same<Team, CtaTeam>::value) car = nrot <= DYN_SMEM / 8 - 2 * DB * (DB + 1);
    if (car) {
      __syncthreads();
      for (int p = tid; p < nrot; p += NT) s_car[p] = ldcg(Rcol(ldcg(I.rslot + q + p)) + q);
    }
    for (int blk = tm.rank; blk < nblk; blk += tm.size) {
      const int bs = q + blk * DB;
      const int bend = min(bs + DB, np - 1);
      const int nown = bend - bs;
      __syncthreads();
      // rows below bs are the only ones earlier rotations touch: stage the
      // block's own rows (bs+1 .. bs+DB) once
      for (int idx = tid; idx < DB * DB; idx += NT) {
        const int l = idx / DB, e = idx - (idx / DB) * DB;
        double v = 0.0;
        if (bs + l < np - 1 && e <= l) v = ldcg(Rcol(ldcg(I.rslot + bs + l)) + bs + 1 + e);
        sB[e * (DB + 1) + l] = v;
      }
      if (tid == 0) {
        *prog = 0;
        *qprog = 0;
      }
      __syncthreads();
      for (int idx = tid; idx < DB * DB; idx += NT) {
        const int e = idx / DB, l = idx - e * DB;
        const double be = sB[e * (DB + 1) + e];
        sY[e * (DB + 1) + l] = (be != 0.0) ? -sB[e * (DB + 1) + l] * rcp_nr(be) : 0.0;
      }
      __syncthreads();
      if (warp == 0) {
        const int pl = bs + lane;
        const bool act = pl < np - 1;
        const double* col = act ? Rcol(ldcg(I.rslot + pl)) : nullptr;
        double carry = act ? (car ? s_car[pl - q] : ldcg(col + q)) : 0.0;
        // the one-FMA form of the block's own steps (below) when every b_e
        // is nonzero and within 2^+-24 (the products of 32 of them stay far
        // inside the FP64 range): Dx = prod_{i < lane} (-b_i)
        const double bme = (lane < nown) ? sB[lane * (DB + 1) + lane] : 1.0;
        const bool fast = __all_sync(0xffffffffu, lane >= nown || (bme != 0.0 && abs(ebound(bme)) < 24));
        double Dx = 1.0;
        if (fast) {
          double Di = (lane < nown) ? -bme : 1.0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const double tt = __shfl_up_sync(0xffffffffu, Di, o);
            if (lane >= o) Di *= tt;
          }
          Dx = __shfl_up_sync(0xffffffffu, Di, 1);
          if (lane == 0) Dx = 1.0;
        }
        // earlier blocks' rotations, as they appear in the log, up to 16 at
        // a time (lanes 0-15 poll cosines, 16-31 sines); the column values
        // are loaded before the wait.  carry = row t of this column after
        // rotations q .. t-1: carry' = -sin carry + cos R(t+1, column).
        int t = car ? bs : q;  // (the one-CTA team's carries are current)
        bool expired = false;
        const long long tw0 = gtimer();
        unsigned spins = 0;
        while (t < bs) {
          const int want = min(16, bs - t);
          double bot[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) bot[e] = (act && e < want) ? ldcg(col + t + 1 + e) : 0.0;
          const int j = lane & 15;
          const double* src = (lane < 16 ? I.rotc : I.rots) + (t - q) + j;
          double rv = 0.0;
          unsigned okm = 0u;
          for (;;) {
            rv = (j < want) ? *(volatile const double*)src : 0.0;
            const unsigned m = __ballot_sync(0xffffffffu, j < want && !isnan(rv));
            okm = m & (m >> 16) & 0xffffu;
            if (okm & 1u) break;
            if ((++spins & 63u) == 0u) {
              int bad = 0;
              if (lane == 0) {
                int* er = tm_err();
                bad = (er && *(volatile int*)er) ? 1 : 0;
                if (!bad && gtimer() - tw0 > I.wait_ns) {
                  if (er) atomicExch(er, 1);
                  bad = 1;
                }
              }
              if (__shfl_sync(0xffffffffu, bad, 0)) { expired = true; break; }
            }
          }
          if (expired) break;
          const int cnt = __ffs(~okm) - 1;  // leading run of published rotations
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            if (e < cnt) {
              const double cs = __shfl_sync(0xffffffffu, rv, e), sn = __shfl_sync(0xffffffffu, rv, 16 + e);
              carry = fma(cs, bot[e], -sn * carry);
            }
          }
          t += cnt;
        }
        if (expired) {
          if (lane == 0) *prog = -1;
          continue;
        }
        // own block, unnormalised.  Lane l keeps xt_l = X_l S_e, X_l the row
        // e value of position bs+l, S_e^2 = Q_e the product of the squared
        // radii of the block's rotations so far (Q_0 = 1).  Rotation e has
        // a~ = xt of lane e (one shuffle) and b = R(t+1, position t); the new
        // row e+1 of lane l is a~ y_l - b xt_l at scale S_{e+1}, with
        // Q_{e+1} = a~^2 + b^2 Q_e formed by the publisher: two FP64
        // instructions per rotation and no square root or division on the
        // chain.  Steps run in groups of RG (the group's b and y read from
        // shared memory first); at a group's end S is renormalised by an exact
        // power of two if the largest |xt| has left [2^-128, 2^128], and
        // a~, the zero-radius flags and the exponent go to the publisher.
        constexpr int RG = 8;
        double xt = carry;
        // One-FMA form: with D_e = prod_{i < e} (-b_i), z_l = xt_l / D_e
        // moves as z_l += z_e Y~(e, l), Y~ = -y / b: one FP64 instruction
        // per step instead of two.  At a group's end a~ = z D of the lane's
        // own step, and the lanes still to come go on at scale D_{el+1}
        // (their xt = z D_{el+1} decides the renormalisation, applied to z
        // as to xt).  No zero radius can occur (b != 0).
        for (int e0 = 0; fast && e0 < nown; e0 += RG) {
          double yg[RG];
#pragma unroll
          for (int jj = 0; jj < RG; ++jj) yg[jj] = sY[min(e0 + jj, DB - 1) * (DB + 1) + lane];
#pragma unroll
          for (int jj = 0; jj < RG; ++jj) {
            const int e = e0 + jj;
            if (e < nown) {
              const double a = __shfl_sync(0xffffffffu, xt, e);
              if (lane > e) xt = fma(a, yg[jj], xt);
            }
          }
          const int el = min(e0 + RG, nown) - 1;
          const bool mine = lane >= e0 && lane <= el;
          const double Dn = __shfl_sync(0xffffffffu, Dx, min(el + 1, DB - 1));
          const double xs = xt * (lane <= el ? Dx : Dn);  // a~ (mine), or xt at scale D_{el+1}
          if (mine) {
            s_ra[lane] = xs;
            s_rid[lane] = 0;
          }
          int ex = (act && lane > el) ? (int)((__double_as_longlong(xs) >> 52) & 0x7ff) : 0;
#pragma unroll
          for (int o = 16; o; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
          int k = 0;
          if (ex > 1023 + 128 || (ex > 0 && ex < 1023 - 128)) {
            k = ex - 1023;
            if (lane > el) xt = ldexp(xt, -k);
          }
          if (mine) s_rk[lane] = (lane == el) ? k : 0;
          __threadfence_block();
          if (lane == 0) *prog = el + 1;
          __syncwarp();
        }
        for (int e0 = 0; !fast && e0 < nown; e0 += RG) {
          double bg[RG], yg[RG];
#pragma unroll
          for (int jj = 0; jj < RG; ++jj) {
            const int e = min(e0 + jj, DB - 1);
            bg[jj] = sB[e * (DB + 1) + e];
            yg[jj] = sB[e * (DB + 1) + lane];
          }
          const double xt0 = xt;
          // lane e stops updating after step e, so at the group's end it
          // still holds its a~
#pragma unroll
          for (int jj = 0; jj < RG; ++jj) {
            const int e = e0 + jj;
            if (e < nown) {
              const double nbx = -bg[jj] * xt;
              const double a = __shfl_sync(0xffffffffu, xt, e);
              if (lane > e) xt = fma(a, yg[jj], nbx);
            }
          }
          const int el = min(e0 + RG, nown) - 1;
          const bool mine = lane >= e0 && lane <= el;
          double my_b = 0.0;
#pragma unroll
          for (int jj = 0; jj < RG; ++jj)
            if (lane == e0 + jj) my_b = bg[jj];
          int my_id = 0;
          const unsigned zm = __ballot_sync(0xffffffffu, mine && xt == 0.0 && my_b == 0.0);
          if (zm) {
            // a zero radius (a~ = b = 0: identity rotation; the rows stay as
            // they are and the scale restarts at 1): redo the group with it
            xt = xt0;
            for (int jj = 0; jj < RG; ++jj) {
              const int e = e0 + jj;
              if (e < nown) {
                const double nbx = -bg[jj] * xt;
                const double a = __shfl_sync(0xffffffffu, xt, e);
                const int idr = (a == 0.0 && bg[jj] == 0.0) ? 1 : 0;
                if (lane > e) xt = idr ? yg[jj] : fma(a, yg[jj], nbx);
                if (lane == e) my_id = idr;
              }
            }
          }
          if (mine) {
            s_ra[lane] = xt;
            s_rid[lane] = my_id;
          }
          // renormalise S: the largest exponent of the lanes whose row is
          // still to be generated
          int ex = (act && lane > el) ? (int)((__double_as_longlong(xt) >> 52) & 0x7ff) : 0;
#pragma unroll
          for (int o = 16; o; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
          int k = 0;
          if (ex > 1023 + 128 || (ex > 0 && ex < 1023 - 128)) {
            k = ex - 1023;
            if (lane > el) xt = ldexp(xt, -k);
          }
          if (mine) s_rk[lane] = (lane == el) ? k : 0;
          __threadfence_block();
          if (lane == 0) *prog = el + 1;
          __syncwarp();
        }
      } else if (warp == 2) {
        // scale: Q_{e+1} = (zero radius ? 1 : a~^2 + b^2 Q_e) 2^(-2k_e) is an
        // affine map of Q_e; each group of RG rotations the generator hands
        // over gets its Q values from a prefix scan of those maps over the
        // group's lanes (the same association whatever the timing)
        constexpr int RG = 8;
        int done = 0;
        double qrun = 1.0;  // Q_done
        const long long tw0 = gtimer();
        unsigned spins = 0;
        while (done < nown) {
          const int pg = __shfl_sync(0xffffffffu, *prog, 0);
          if (pg < 0) {
            if (lane == 0) *qprog = -1;
            break;
          }
          const int gend = min(done + RG, nown);
          if (pg >= gend) {
            __threadfence_block();
            const int k = done + lane;
            const bool in = k < gend;
            const double a = in ? s_ra[k] : 0.0, bk = in ? sB[k * (DB + 1) + k] : 0.0;
            const int idr = in ? s_rid[k] : 0, rk = in ? s_rk[k] : 0;
            const double sc = (rk != 0) ? ldexp(1.0, -2 * rk) : 1.0;
            double Cm = in ? (idr ? sc : (a * a) * sc) : 0.0;
            double Dm = in ? (idr ? 0.0 : (bk * bk) * sc) : 1.0;
#pragma unroll
            for (int o = 1; o < RG; o <<= 1) {
              const double Cp = __shfl_up_sync(0xffffffffu, Cm, o);
              const double Dp = __shfl_up_sync(0xffffffffu, Dm, o);
              if (lane >= o) {
                Cm = fma(Dm, Cp, Cm);
                Dm = Dm * Dp;
              }
            }
            const double qnext = fma(Dm, qrun, Cm);  // Q_{k+1}
            double qk = __shfl_up_sync(0xffffffffu, qnext, 1);
            if (lane == 0) qk = qrun;                // Q_k
            if (in) {
              s_rq[k] = qk;
              s_rqa[k] = idr ? 1.0 : fma(a, a, (bk * bk) * qk);
            }
            qrun = __shfl_sync(0xffffffffu, qnext, gend - done - 1);
            __threadfence_block();
            if (lane == 0) *qprog = gend;
            __syncwarp();
            done = gend;
          } else if ((++spins & 63u) == 0u) {
            int bad = 0;
            if (lane == 0) {
              int* er = tm_err();
              bad = (er && *(volatile int*)er) ? 1 : 0;
              if (!bad && gtimer() - tw0 > I.wait_ns) {
                if (er) atomicExch(er, 1);
                bad = 1;
              }
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) {
              if (lane == 0) *qprog = -1;
              break;
            }
          }
        }
      } else if (warp == 1) {
        // publish cos = a~ / S_{e+1} and sin = b S_e / S_{e+1} (identity for a
        // zero radius), one rotation per lane, as the scale warp hands them
        // over
        int done = 0;
        const long long tw0 = gtimer();
        unsigned spins = 0;
        while (done < nown) {
          const int pg = __shfl_sync(0xffffffffu, *qprog, 0);
          if (pg < 0) break;
          if (pg > done) {
            __threadfence_block();
            const int k = done + lane;
            if (k < pg) {
              const double a = s_ra[k], bk = sB[k * (DB + 1) + k], qk = s_rq[k], qa = s_rqa[k];
              const bool idr = s_rid[k] != 0;
              const double iqa = idr ? 0.0 : rsqrt(qa);
              I.rots[bs - q + k] = idr ? 0.0 : bk * sqrt_gm(qk) * iqa;
              I.rotc[bs - q + k] = idr ? 1.0 : a * iqa;
            }
            done = pg;
          } else if ((++spins & 63u) == 0u) {
            int bad = 0;
            if (lane == 0) {
              int* er = tm_err();
              bad = (er && *(volatile int*)er) ? 1 : 0;
              if (!bad && gtimer() - tw0 > I.wait_ns) {
                if (er) atomicExch(er, 1);
                bad = 1;
              }
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) break;
          }
        }
      }
      if (car && bend < np - 1) {
        // the later positions' row values through this block's rotations:
        // carry' = -sin carry + cos R(t+1, column), t = bs .. bend-1
        __syncthreads();
        if (tid < nown) {
          s_rc[tid] = ldcg(I.rotc + bs - q + tid);
          s_rs[tid] = ldcg(I.rots + bs - q + tid);
        }
        __syncthreads();
        for (int p = bend + tid; p < np - 1; p += NT) {
          const double* col = Rcol(ldcg(I.rslot + p));
          double c = s_car[p - q];
          for (int t0 = 0; t0 < nown; t0 += 8) {
            double bot[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) bot[e] = (t0 + e < nown) ? ldcg(col + bs + 1 + t0 + e) : 0.0;
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (t0 + e < nown) c = fma(s_rc[t0 + e], bot[e], -s_rs[t0 + e] * c);
          }
          s_car[p - q] = c;
        }
      }
    }
    if (follow && tm.rank >= nblk && !rotate_columns(q, np, nrot, nblk, true)) {
      failed = true;
      status = LHDM_ERR_TIMEOUT;
      return false;
    }
    if (!sync()) return false;
    phase(PH_ZROT);
    nP = np - 1;
    if (!follow) rotate_columns(q, np, nrot, 0, false);
    const bool ok = sync();
    phase(PH_INNER);
    return ok;
  }

  // (ii) of the downdate: the rotations on every Z column and on b, and on
  // R's columns at positions q .. np-2 (rows q .. p+1 of position p take
  // rotations q .. p; the last one zeroes row p+1): one warp per column; the
  // carry recurrence c' = -s c + cs * bot is affine, so each 32-row chunk is
  // a warp-wide prefix scan of affine maps.  Ranks r0 .. size-1 share the
  // columns.  With `follow` (ranks the chain leaves free, all rotations in
  // one shared-memory stage) the work runs while the chain is still
  // generating: warp 0 stages each 32-rotation chunk of the log as it is
  // published and the other warps follow it; an R column starts once its
  // own chain block's rotations are out, when that block no longer reads it
  // (the chain never reads W or b).
  __device__ bool rotate_columns(int q, int np, int nrot, int r0rank, bool follow) {
    static_assert(DB == 32, "a chain block's rotations are one 32-rotation chunk");
    double* s_c = dyn;
    double* s_s = dyn + ROT_STAGE;
    // the scan's multiplicative parts, the same for every column: per
    // 32-rotation chunk, lane t's running product of -sin before each of
    // the five levels (rows 0-4) and after the last (row 5)
    double* s_am = dyn + 2 * ROT_STAGE;  // 6 x ROT_STAGE
    const int zr = tm.rank - r0rank, nzr = tm.size - r0rank;
    int c0, c1;
    split(I.n, nzr, zr, c0, c1);
    const bool do_b = (zr == nzr - 1);
    __shared__ int s_zl[CAND_LOCAL_MAX + 1];
    __shared__ int s_nz, s_avail;
    volatile int* avail = &s_avail;  // chunks staged (follow); -1: abandoned
    if (tid == 0) {
      s_nz = 0;
      s_avail = 0;
    }
    __syncthreads();
    for (int c = c0 + tid; c < c1; c += NT)
      if (ldcg(I.pos + c) < 0) s_zl[atomicAdd(&s_nz, 1)] = c;
    __syncthreads();
    const int nz = s_nz + (do_b ? 1 : 0);
    // R columns round-robin over the ranks (the last positions, which take
    // the most rotations, land on different CTAs)
    const int nr_own = (zr < nrot) ? (nrot - zr + nzr - 1) / nzr : 0;
    const int nunit = nz + nr_own;
    // the products for the chunk at stage offset t0 (one warp)
    auto chunk_products = [&](int t0, int ns) {
      const int cnt = min(32, ns - t0);
      double Am = (lane < cnt) ? -s_s[t0 + lane] : 1.0;
#pragma unroll
      for (int lv = 0; lv < 5; ++lv) {
        s_am[lv * ROT_STAGE + t0 + lane] = Am;
        const double Ap = __shfl_up_sync(0xffffffffu, Am, 1 << lv);
        if (lane >= (1 << lv)) Am *= Ap;
      }
      s_am[5 * ROT_STAGE + t0 + lane] = Am;
    };
    // rotations rb + t0 .. rb + t0 + cnt - 1 (stage offset t0) on one column
    auto chunk_apply = [&](double* colp, int rb, int t0, int cnt, double bot, double& carry) {
      double cs = 1.0, sn = 0.0;
      if (lane < cnt) {
        cs = s_c[t0 + lane];
        sn = s_s[t0 + lane];
      }
      // lanes past cnt may hold other rotations' products: no lane below
      // cnt reads them
      double Bm = (lane < cnt) ? cs * bot : 0.0;
#pragma unroll
      for (int lv = 0; lv < 5; ++lv) {
        const double Bp = __shfl_up_sync(0xffffffffu, Bm, 1 << lv);
        if (lane >= (1 << lv)) Bm = fma(s_am[lv * ROT_STAGE + t0 + lane], Bp, Bm);
      }
      const double incl = fma(s_am[5 * ROT_STAGE + t0 + lane], carry, Bm);  // carry after rotation lane
      double cin = __shfl_up_sync(0xffffffffu, incl, 1);
      if (lane == 0) cin = carry;
      if (lane < cnt) colp[q + rb + t0 + lane] = cs * cin + sn * bot;
      carry = __shfl_sync(0xffffffffu, incl, cnt - 1);
    };
    // unit k: its column, its rotation count from rb on, whether they end an
    // R column's rotations
    auto unit = [&](int k, int rb, int ns, double*& colp, int& nsu, bool& rlast) {
      nsu = ns;
      rlast = false;
      if (k < nz) {
        colp = (k < s_nz) ? Wcol(s_zl[k]) : I.bt;
      } else {
        const int pr = q + zr + (k - nz) * nzr;  // R column at position pr
        colp = Rcol(ldcg(I.rslot + pr));
        nsu = min(ns, pr - q + 1 - rb);
        rlast = (rb + nsu == pr - q + 1);
      }
    };
    // a column's last carry: zero below an R column's diagonal; for a Z
    // column row np-1 joins the trailing part and its norm grows by that
    // entry (an update, free of cancellation)
    auto finish_unit = [&](int k, double* colp, int at, bool rlast, double carry, bool last) {
      if (lane == 0) {
        colp[at] = rlast ? 0.0 : carry;
        if (last && k < s_nz) {
          const int c = s_zl[k];
          const double uo = ldcg(I.u + c);
          I.u[c] = sqrt(fma(carry, carry, uo * uo));
        }
      }
    };
    bool ok = true;
    bool lanes = false;
    if constexpr (std::is_same<Team, CtaTeam>::value) lanes = nrot > 0 && nrot <= ROT_STAGE;
    if (lanes) {
      // One CTA holds every column, so a lane can take a whole column: the
      // recurrence runs down the rows one rotation at a time, four FP64
      // instructions per 32 columns and rotation against the scan's nine
      // per 32 rows of one column.  Columns go in groups of 32 per warp (Z
      // columns and b first, then R's, whose rotation counts grow by one per
      // position); 16-rotation row tiles of the group are staged in shared
      // memory with coalesced loads (a column's 16 rows per half-warp) and
      // written back the same way.
      constexpr int TR = 16;
      double* sT = dyn + 2 * ROT_STAGE + warp * (TR * 33);
      __syncthreads();
      for (int e = tid; e < nrot; e += NT) {
        s_c[e] = ldcg(I.rotc + e);
        s_s[e] = ldcg(I.rots + e);
      }
      __syncthreads();
      const int ncol = nz + nrot;
      for (int g = warp; g * 32 < ncol; g += NW) {
        const int k = g * 32 + lane;
        double* colp = I.bt;
        int nsu = 0;
        bool rlast = false;
        if (k < ncol) unit(k, 0, nrot, colp, nsu, rlast);
        double carry = (nsu > 0) ? ldcg(colp + q) : 0.0;
        int gmax = nsu;
#pragma unroll
        for (int o = 16; o; o >>= 1) gmax = max(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        const int hl = lane >> 4, il = lane & 15;
        for (int t0 = 0; t0 < gmax; t0 += TR) {
          // rows q+t0+1 .. q+t0+TR (the bots of rotations t0 ..)
          for (int cc = 0; cc < 32; cc += 2) {
            const int c = cc + hl;
            const double* cp = reinterpret_cast<const double*>(__shfl_sync(0xffffffffu, reinterpret_cast<long long>(colp), c));
            const int ns_c = __shfl_sync(0xffffffffu, nsu, c);
            sT[il * 33 + c] = (t0 + il < ns_c) ? ldcg(cp + q + t0 + 1 + il) : 0.0;
          }
          __syncwarp();
#pragma unroll 4
          for (int i = 0; i < TR; ++i) {
            const int t = t0 + i;
            if (t < nsu) {
              const double cs = s_c[t], sn = s_s[t], bot = sT[i * 33 + lane];
              const double out = fma(sn, bot, cs * carry);
              carry = fma(cs, bot, -sn * carry);
              sT[i * 33 + lane] = out;
            }
          }
          __syncwarp();
          // outputs of rotations t0 .. go to rows q+t0 ..
          for (int cc = 0; cc < 32; cc += 2) {
            const int c = cc + hl;
            double* cp = reinterpret_cast<double*>(__shfl_sync(0xffffffffu, reinterpret_cast<long long>(colp), c));
            const int ns_c = __shfl_sync(0xffffffffu, nsu, c);
            if (t0 + il < ns_c) cp[q + t0 + il] = sT[il * 33 + c];
          }
          __syncwarp();
        }
        if (nsu > 0) {
          colp[q + nsu] = rlast ? 0.0 : carry;
          if (k < s_nz) {
            const int c = s_zl[k];
            const double uo = ldcg(I.u + c);
            I.u[c] = sqrt(fma(carry, carry, uo * uo));
          }
        }
      }
    } else if (!follow) {
      for (int rb = 0; rb < nrot; rb += ROT_STAGE) {
        const int ns = min(ROT_STAGE, nrot - rb);
        __syncthreads();
        for (int e = tid; e < ns; e += NT) {
          s_c[e] = ldcg(I.rotc + rb + e);
          s_s[e] = ldcg(I.rots + rb + e);
        }
        __syncthreads();
        for (int t0 = warp * 32; t0 < ns; t0 += NW * 32) chunk_products(t0, ns);
        __syncthreads();
        for (int k = warp; k < nunit; k += NW) {
          double* colp;
          int nsu;
          bool rlast;
          unit(k, rb, ns, colp, nsu, rlast);
          if (nsu <= 0) continue;
          double carry = ldcg(colp + q + rb);
          // next chunk's column values are loaded before the scan of this one
          double nbot = (lane < nsu) ? ldcg(colp + q + rb + 1 + lane) : 0.0;
          for (int t0 = 0; t0 < nsu; t0 += 32) {
            const double bot = nbot;
            nbot = (t0 + 32 + lane < nsu) ? ldcg(colp + q + rb + t0 + 33 + lane) : 0.0;
            chunk_apply(colp, rb, t0, min(32, nsu - t0), bot, carry);
          }
          finish_unit(k, colp, q + rb + nsu, rlast, carry, rb + ns == nrot);
        }
      }
      if (nrot == 0) {
        // the last position went: row np-1 joins the trailing part unrotated
        for (int k = tid; k < s_nz; k += NT) {
          const int c = s_zl[k];
          const double v = ldcg(Wcol(c) + np - 1), uo = ldcg(I.u + c);
          I.u[c] = sqrt(fma(v, v, uo * uo));
        }
      }
    } else if (warp == 0) {
      // stage the log chunk by chunk as it is published (every slot holds
      // NaN until its rotation is written)
      const int nch = (nrot + 31) / 32;
      const long long tw0 = gtimer();
      unsigned spins = 0;
      for (int ch = 0; ch < nch && ok; ++ch) {
        const int t = ch * 32 + lane;
        const bool in = t < nrot;
        double cv = 1.0, sv = 0.0;
        for (;;) {
          if (in) {
            cv = *(volatile const double*)(I.rotc + t);
            sv = *(volatile const double*)(I.rots + t);
          }
          if (__ballot_sync(0xffffffffu, in && (isnan(cv) || isnan(sv))) == 0u) break;
          __nanosleep(200);  // the generating CTAs poll the same lines
          if ((++spins & 63u) == 0u) {
            int bad = 0;
            if (lane == 0) {
              int* er = tm_err();
              bad = (er && *(volatile int*)er) ? 1 : 0;
              if (!bad && gtimer() - tw0 > I.wait_ns) {
                if (er) atomicExch(er, 1);
                bad = 1;
              }
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) {
              ok = false;
              break;
            }
          }
        }
        if (!ok) break;
        if (in) {
          s_c[t] = cv;
          s_s[t] = sv;
        }
        __syncwarp();
        chunk_products(ch * 32, nrot);
        __threadfence_block();
        __syncwarp();
        if (lane == 0) *avail = ch + 1;
      }
      if (!ok && lane == 0) *avail = -1;
    } else {
      // wait until n chunks are staged (false: abandoned or timed out)
      auto wait_avail = [&](int n) {
        int st = 0;
        if (lane == 0) {
          const long long tw0 = gtimer();
          unsigned spins = 0;
          for (;;) {
            const int a = *avail;
            if (a < 0) { st = 0; break; }
            if (a >= n) { st = 1; break; }
            if ((++spins & 63u) == 0u && gtimer() - tw0 > I.wait_ns) {
              int* er = tm_err();
              if (er) atomicExch(er, 1);
              st = 0;
              break;
            }
          }
        }
        st = __shfl_sync(0xffffffffu, st, 0);
        __threadfence_block();
        return st != 0;
      };
      for (int k = warp - 1; k < nunit && ok; k += NW - 1) {
        double* colp;
        int nsu;
        bool rlast;
        unit(k, 0, nrot, colp, nsu, rlast);
        // an R column waits for its own chain block's rotations: that block
        // read the column from global memory before generating them
        if (k >= nz && !wait_avail((nsu - 1) / DB + 1)) {
          ok = false;
          break;
        }
        double carry = ldcg(colp + q);
        double nbot = (lane < nsu) ? ldcg(colp + q + 1 + lane) : 0.0;
        for (int t0 = 0; t0 < nsu; t0 += 32) {
          if (!wait_avail(t0 / 32 + 1)) {
            ok = false;
            break;
          }
          const double bot = nbot;
          nbot = (t0 + 32 + lane < nsu) ? ldcg(colp + q + t0 + 33 + lane) : 0.0;
          chunk_apply(colp, 0, t0, min(32, nsu - t0), bot, carry);
        }
        if (!ok) break;
        finish_unit(k, colp, q + nsu, rlast, carry, true);
      }
    }
    // the triangular solve that follows reads rhs = (Q^T b)[0:np-1]
    if (__syncthreads_or(!ok)) return false;
    if (do_b)
      for (int p = tid; p < np - 1; p += NT) I.rhs[p] = ldcg(I.bt + p);
    return true;
  }

  __device__ int* tm_err();

  // ------------------------------------------------------------ residual and dual
  // r = b - A_P x_P (row tiles of 32 rows, warps split the positions).
  __device__ void residual() {
    __shared__ double s_acc[NW][32];
    double rs = 0.0;
    const int ntile = (I.m + 31) / 32;
    // the passive order and y_P, staged once if they fit (else read from L2)
    const bool staged = (size_t)nP * 12 + 16 <= (size_t)DYN_SMEM && tm.rank < ntile;
    double* s_yv = dyn;
    int* s_ov = reinterpret_cast<int*>(dyn + nP);
    if (staged) {
      for (int p = tid; p < nP; p += NT) {
        s_yv[p] = ldcg(I.yP + p);
        s_ov[p] = ldcg(I.order + p);
      }
      __syncthreads();
    }
    for (int tile = tm.rank; tile < ntile; tile += tm.size) {
      const int row = tile * 32 + lane;
      double acc = 0.0, acc2 = 0.0;
      if (row < I.m) {
        int p = warp;
        if (staged) {
          // eight columns' loads in flight per lane
          for (; p + 7 * NW < nP; p += 8 * NW) {
            double av[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) av[j] = __ldg(I.A + (size_t)s_ov[p + j * NW] * I.lda + row);
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              acc = fma(av[j], s_yv[p + j * NW], acc);
              acc2 = fma(av[j + 1], s_yv[p + (j + 1) * NW], acc2);
            }
          }
          for (; p < nP; p += NW) acc = fma(__ldg(I.A + (size_t)s_ov[p] * I.lda + row), s_yv[p], acc);
        } else {
          for (; p + NW < nP; p += 2 * NW) {
            const int c = ldcg(I.order + p), c2 = ldcg(I.order + p + NW);
            acc = fma(__ldg(I.A + (size_t)c * I.lda + row), ldcg(I.yP + p), acc);
            acc2 = fma(__ldg(I.A + (size_t)c2 * I.lda + row), ldcg(I.yP + p + NW), acc2);
          }
          for (; p < nP; p += NW) {
            const int c = ldcg(I.order + p);
            acc = fma(__ldg(I.A + (size_t)c * I.lda + row), ldcg(I.yP + p), acc);
          }
        }
      }
      s_acc[warp][lane] = acc + acc2;
      __syncthreads();
      if (warp == 0 && row < I.m) {
        double s = 0.0;
        for (int k = 0; k < NW; ++k) s += s_acc[k][lane];
        const double rv = __ldg(I.b + row) - s;
        I.r[row] = rv;
        rs = fma(rv, rv, rs);
      }
      __syncthreads();
    }
    // x = y on P
    const int gt = tm.rank * NT + tid, nt = tm.size * NT;
    for (int p = gt; p < nP; p += nt) I.xP[p] = ldcg(I.yP + p);
    __shared__ double sh[32];
    rs = block_sum(rs, sh);
    if (tid == 0) I.part[(size_t)tm.rank * PW + P_RS] = rs;
  }

  // w = A^T r on Z (w_P = 0) and the O1 partial.  The Z columns are split
  // evenly over the team (z_share) and r is staged in shared memory; the
  // CTA's nl x m elements, in column order, are split evenly over its warps
  // (one FP64 instruction per warp is 64 cycles on this GPU whatever the
  // active lanes, so equal shares keep every sub-partition's FP64 pipe busy
  // to the end).  A column inside one warp's share is summed by that warp; a
  // column cut by share boundaries gets its partial sums added in warp
  // order.  The trailing norms u need no pass here: the downdate updates
  // them as it moves a row into the trailing part.
  static constexpr int DUAL_RMAX = 16384;  // rows of r held in shared memory
  __device__ void dual() {
    {
      int c0, c1;
      split(I.n, tm.size, tm.rank, c0, c1);
      for (int c = c0 + tid; c < c1; c += NT)
        if (ldcg(I.pos + c) >= 0) I.w[c] = 0.0;
    }
    const int m = I.m;
    const bool r_in_smem = m <= DUAL_RMAX &&
                           (size_t)m * 8 + (CAND_LOCAL_MAX + 2) * 4 + 8 * (size_t)((I.n + 31) / 32) <= (size_t)DYN_SMEM;
    double* s_r = dyn;                                    // m doubles
    int* s_zl = reinterpret_cast<int*>(dyn + (r_in_smem ? m : 0));
    unsigned* scr = reinterpret_cast<unsigned*>(s_zl + CAND_LOCAL_MAX + 2);
    __shared__ double s_pp[NW][2];  // partial sums of a warp's first and last column
    const int nl = z_share(s_zl, scr, nullptr, 0, false);
    if (r_in_smem)
      for (int i = tid; i < m; i += NT) s_r[i] = ldcg(I.r + i);
    __syncthreads();
    const double* rv = r_in_smem ? s_r : I.r;
    const long long E = (long long)nl * m;
    {
      const long long e0 = E * warp / NW, e1 = E * (warp + 1) / NW;
      if (e0 < e1) {
        const int kf = (int)(e0 / m), kl = (int)((e1 - 1) / m);
        for (int k = kf; k <= kl; ++k) {
          const int i0 = (k == kf) ? (int)(e0 - (long long)k * m) : 0;
          const int i1 = (k == kl) ? (int)(e1 - (long long)k * m) : m;
          const double* a = I.A + (size_t)s_zl[k] * I.lda;
          double s0 = 0.0, s1 = 0.0;
          int i = i0 + lane;
          for (; i + 224 < i1; i += 256) {
            double av[8], rr[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              av[j] = __ldg(a + i + 32 * j);
              rr[j] = r_in_smem ? rv[i + 32 * j] : ldcg(rv + i + 32 * j);
            }
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              s0 = fma(av[j], rr[j], s0);
              s1 = fma(av[j + 1], rr[j + 1], s1);
            }
          }
          for (; i < i1; i += 32) s0 = fma(__ldg(a + i), r_in_smem ? rv[i] : ldcg(rv + i), s0);
          const double tot = warp_sum(s0 + s1);
          if (lane == 0) {
            if (k == kf) s_pp[warp][0] = tot;
            else if (k == kl) s_pp[warp][1] = tot;
            else I.w[s_zl[k]] = tot;
          }
        }
      }
    }
    __syncthreads();
    for (int k = tid; k < nl; k += NT) {
      const long long cs = (long long)k * m, ce = cs + m;
      double sum = 0.0;
      bool direct = false;
      for (int w = 0; w < NW; ++w) {
        const long long a0 = E * w / NW, a1 = E * (w + 1) / NW;
        if (a0 >= a1 || a1 <= cs || a0 >= ce) continue;
        const int kf = (int)(a0 / m), kl = (int)((a1 - 1) / m);
        if (k != kf && k != kl) {
          direct = true;  // written by warp w
          break;
        }
        sum += (k == kf) ? s_pp[w][0] : s_pp[w][1];
      }
      if (!direct) I.w[s_zl[k]] = sum;
    }
    // resid sum of squares of this CTA is in part[PW-1]; fold it into slot 6
    const double rs = ldcg(I.part + (size_t)tm.rank * PW + P_RS);
    o1_partial(0.0, rs, 0.0, s_zl, nl);
  }

  // ------------------------------------------------------------ outputs
  __device__ bool finish() {
    __shared__ int shi[32];
    // x and the sorted passive set.  With the positivity trick x has 2n
    // entries (x+, x-) and the passive set lists indices of [A -A]: every
    // CTA counts its passive columns of either sign, so that the +1 columns
    // come first (index j) and the -1 columns after them (index n + j).
    int c0, c1;
    split(I.n, tm.size, tm.rank, c0, c1);
    int cnt = 0, cneg = 0;
    for (int c = c0 + tid; c < c1; c += NT) {
      const int p = ldcg(I.pos + c);
      const double v = (p >= 0 && status != LHDM_ERR_NONFINITE) ? ldcg(I.xP + p) : 0.0;
      if (!sgn) {
        I.x_out[c] = v;
        cnt += (p >= 0);
      } else {
        const int sc = (p >= 0) ? ldcg(I.csign + c) : 0;
        I.x_out[c] = sc > 0 ? v : 0.0;
        I.x_out[I.n + c] = sc < 0 ? -v : 0.0;
        cnt += (sc > 0);
        cneg += (sc < 0);
      }
    }
    cnt = block_sum_int(cnt, shi);
    cneg = block_sum_int(cneg, shi);
    if (tid == 0) {
      I.ipart[tm.rank * 8] = cnt;
      I.ipart[tm.rank * 8 + 1] = cneg;
    }
    if (!sync()) return false;
    __shared__ int s_base, s_bneg;
    if (tid == 0) {
      int acc = 0, accn = 0, tot = 0;
      for (int t = 0; t < tm.size; ++t) {
        const int ct = ldcg(I.ipart + t * 8);
        if (t < tm.rank) {
          acc += ct;
          accn += ldcg(I.ipart + t * 8 + 1);
        }
        tot += ct;
      }
      s_base = acc;
      s_bneg = tot + accn;
    }
    __syncthreads();
    if (tid == 0) {
      int k = s_base, kn = s_bneg;
      for (int c = c0; c < c1; ++c) {
        if (ldcg(I.pos + c) < 0) continue;
        if (sgn && ldcg(I.csign + c) < 0) I.passive_out[kn++] = I.n + c;
        else I.passive_out[k++] = c;
      }
    }
    const int gt = tm.rank * NT + tid, nt = tm.size * NT;
    for (int p = nP + gt; p < nx; p += nt) I.passive_out[p] = -1;
    if (tm.rank == 0 && tid == 0) {
      lhdm_info inf;
      inf.status = status;
      inf.n_outer = n_outer;
      inf.n_inner = n_inner;
      inf.n_drop = n_drop;
      inf.n_passive = nP;
      inf.rank_limited = rank_limited;
      inf.n_flip = n_flip;
      inf.mode = sgn;
      inf.resid_norm = sqrt(rsq);
      inf.max_wZ = wz_any;
      inf.tol_w = tol_w;
      *I.info_out = inf;
      *I.nP_out = nP;
      if (I.phase_ns) {
        phase(-1);
        for (int i = 0; i < NPHASE; ++i) {
          I.phase_ns[i] = phf[i];
          I.phase_ns[NPHASE + i] = phf[NPHASE + i];
        }
      }
    }
    return true;
  }

  // ------------------------------------------------------------ the solve
  __device__ __forceinline__ void run() {
    phase(PH_SETUP);
    setup();
    flops(PH_SETUP, 4.0 * (double)I.m * I.n);
    if (!sync()) return fail_out();
    o1_reduce(true);
    tol_w = (I.prm.tol_w >= 0.0) ? I.prm.tol_w
                                 : 10.0 * EPS * (double)max(I.m, nx) * amax * sqrt(bsq);
    if (nonfinite) {
      status = LHDM_ERR_NONFINITE;
      nP = 0;
      for (int c = tm.rank * NT + tid; c < I.n; c += tm.size * NT) I.pos[c] = -1;
      if (!sync()) return fail_out();
      finish();
      return;
    }
    __shared__ int s_J[KM];
    const int max_outer = I.prm.max_outer > 0 ? I.prm.max_outer : 3 * nx;
    for (;;) {
      if (n_elig == 0 || !(wmax > tol_w)) {
        if (wz_any > tol_w) rank_limited = 1;
        break;
      }
      if (n_outer >= max_outer) {
        status = LHDM_ERR_MAX_ITER;
        break;
      }
      phase(PH_DM);
      if (!dm_select(s_J)) return fail_out();
      kdm = kk;
      phase(PH_PANEL);
      {
        // the shared-memory panel runs on about Lp / PANEL_ROWS CTAs: its
        // exchanges then move far fewer partial sums
        const int Lp = I.m - nP;
        const int P = min(tm.size, max(1, (Lp + PANEL_ROWS - 1) / PANEL_ROWS));
        const bool in_smem = (Lp + P - 1) / P <= PR_MAX;
        if (!(in_smem ? panel_smem(s_J, P) : panel(s_J))) return fail_out();
      }
      if (kk == 0) {
        rank_limited = 1;
        break;
      }
      phase(PH_FEAS);
      if (!feasibility(s_J)) return fail_out();
      phase(PH_SOLVE);
      // y_P: rhs = (Q^T b)[0:nP] - R12 y_J, then back substitution
      {
        __shared__ double s_yj[KM];
        if (tid < kp) s_yj[tid] = ldcg(I.yJ + tid);
        __syncthreads();
        const int gt = tm.rank * NT + tid, nt = tm.size * NT;
        for (int p = gt; p < nP; p += nt) {
          double s = ldcg(I.bt + p);
          for (int t = 0; t < kp; ++t) s = fma(-ldcg(Wcol(s_J[t]) + p), s_yj[t], s);
          I.rhs[p] = s;
        }
      }
      flops(PH_SOLVE, 2.0 * nP * (double)kp + (double)kk * kk);
      if (!sync()) return fail_out();
      if (!trsv(nP)) return fail_out();
      phase(PH_COMMIT);
      if (!commit(s_J)) return fail_out();
      phase(PH_INNER);
      removed = 0;
      inner_step = 0;
      if (!inner_loop()) return fail_out();
      if (status != LHDM_OK) break;
      phase(PH_RESID);
      flops(PH_RESID, 2.0 * (double)I.m * nP);
      residual();
      if (!sync()) return fail_out();
      phase(PH_DUAL);
      flops(PH_DUAL, 2.0 * (double)I.m * (double)(I.n - nP));
      dual();
      if (!sync()) return fail_out();
      if (I.trace && tm.rank == 0 && tid == 0 && n_outer < I.trace_cap) {
        int* tr = I.trace + 6 * n_outer;
        tr[0] = kdm;
        tr[1] = kp;
        tr[2] = inner_step;
        tr[3] = nP;
        tr[4] = removed;
        tr[5] = jsel;  // the first column of J (its index in [A -A] with the positivity trick)
      }
      o1_reduce(false);
      ++n_outer;
    }
    phase(PH_SETUP);
    finish();
  }

  __device__ void fail_out() {
    // a bounded wait expired: report and leave without further barriers
    if (tm.rank == 0 && tid == 0) {
      lhdm_info inf;
      inf.status = LHDM_ERR_TIMEOUT;
      inf.n_outer = n_outer;
      inf.n_inner = n_inner;
      inf.n_drop = n_drop;
      inf.n_passive = nP;
      inf.rank_limited = rank_limited;
      inf.n_flip = n_flip;
      inf.mode = sgn;
      inf.resid_norm = -1.0;
      inf.max_wZ = 0.0;
      inf.tol_w = tol_w;
      *I.info_out = inf;
      *I.nP_out = 0;
    }
  }
};

template <>
__device__ __forceinline__ int* Engine<GridTeam>::tm_err() { return tm.err; }
template <>
__device__ __forceinline__ int* Engine<CtaTeam>::tm_err() { return nullptr; }

}  // namespace lhdm
