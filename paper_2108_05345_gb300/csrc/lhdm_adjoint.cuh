// lhdm_adjoint.cuh -- adjoint of the NNLS solution map on the final passive
// set, reusing the R factor the solve left behind.
//
// On a fixed passive set P the solution is the least-squares solution on P
// (subproblem (6) of section 2.1), x_P = (A_P^T A_P)^{-1} A_P^T b.  With
// g = dL/dx, u = (R^T R)^{-1} g_P and r = b - A x:
//   dL/db   = A_P u
//   dL/dA_P = r u^T - (A_P u) x_P^T,   dL/dA_Z = 0.
// R^T v = g_P is a blocked forward substitution, R u = v the back
// substitution of the solve (Engine::trsv).
#pragma once

#include "lhdm_solve.cuh"

namespace lhdm {

template <class Team>
struct Adjoint {
  Engine<Team>& E;
  const Inst& I;
  int tid, lane, warp;
  __device__ Adjoint(Engine<Team>& e) : E(e), I(e.I) {
    tid = threadIdx.x;
    lane = tid & 31;
    warp = tid >> 5;
  }

  // R^T v = rhs on positions [0, np); result in yP (blocked forward
  // substitution, one barrier per TB-block).
  __device__ bool trsv_t(int np) {
    if (np <= 0) return true;
    const int nb = (np + TB - 1) / TB;
    __shared__ double s_y[TB];
    __shared__ double s_r[TB];
    for (int bi = 0; bi < nb; ++bi) {
      const int b0 = bi * TB, b1 = min(np, b0 + TB);
      const bool has_prev = bi > 0;
      const int c0 = b0 - TB, c1 = b0;
      if (has_prev) {
        if (tid < c1 - c0) s_y[tid] = ldcg(I.yP + c0 + tid);
        __syncthreads();
        // rows (columns of R) [b1, np): contribution of block bi-1
        const int gt = E.tm.rank * NT + tid, nt = E.tm.size * NT;
        for (int row = b1 + gt; row < np; row += nt) {
          const double* col = E.Rcol(ldcg(I.rslot + row));
          double s = 0.0;
          for (int j = 0; j < c1 - c0; ++j) s = fma(ldcg(col + c0 + j), s_y[j], s);
          I.rhs[row] = ldcg(I.rhs + row) - s;
        }
      }
      if (E.tm.rank == 0) {
        if (tid < b1 - b0) {
          double s = ldcg(I.rhs + b0 + tid);
          if (has_prev) {
            const double* col = E.Rcol(ldcg(I.rslot + b0 + tid));
            for (int j = 0; j < c1 - c0; ++j) s = fma(-ldcg(col + c0 + j), s_y[j], s);
          }
          s_r[tid] = s;
        }
        __syncthreads();
        if (warp == 0) {
          // lane holds rows b0+lane, b0+lane+32; column i of R^T is row i of R
          double a0 = (lane < b1 - b0) ? s_r[lane] : 0.0;
          double a1 = (lane + 32 < b1 - b0) ? s_r[lane + 32] : 0.0;
          const double* c0p = (lane < b1 - b0) ? E.Rcol(ldcg(I.rslot + b0 + lane)) : nullptr;
          const double* c1p = (lane + 32 < b1 - b0) ? E.Rcol(ldcg(I.rslot + b0 + lane + 32)) : nullptr;
          for (int jj = 0; jj < b1 - b0; ++jj) {
            const int owner = jj & 31;
            const bool hi = jj >= 32;
            double yv = 0.0;
            if (lane == owner) {
              const double* cp = hi ? c1p : c0p;
              yv = (hi ? a1 : a0) / ldcg(cp + b0 + jj);
            }
            yv = __shfl_sync(0xffffffffu, yv, owner);
            if (lane == owner) I.yP[b0 + jj] = yv;
            // rows i > jj: R^T[i, jj] = R[jj, i] = column i at row b0+jj
            if (lane > jj && c0p) a0 -= ldcg(c0p + b0 + jj) * yv;
            if (lane + 32 > jj && c1p) a1 -= ldcg(c1p + b0 + jj) * yv;
          }
        }
      }
      if (!E.sync()) return false;
    }
    return true;
  }

  __device__ bool run(const double* g, double* dLdb, double* dLdA, int ld_dA, double* apu) {
    const int np = ldcg(I.nP_out);
    E.nP = np;
    // rhs = g_P (position order); pos rebuilt from the persistent order
    {
      const int gt = E.tm.rank * NT + tid, nt = E.tm.size * NT;
      for (int p = gt; p < np; p += nt) I.rhs[p] = __ldg(g + ldcg(I.order + p));
      for (int c = gt; c < I.n; c += nt) I.pos[c] = -1;
    }
    E.clear_tri_flags();
    if (!E.sync()) return false;
    {
      const int gt = E.tm.rank * NT + tid, nt = E.tm.size * NT;
      for (int p = gt; p < np; p += nt) I.pos[ldcg(I.order + p)] = p;
    }
    if (!trsv_t(np)) return false;                 // v in yP
    {
      const int gt = E.tm.rank * NT + tid, nt = E.tm.size * NT;
      for (int p = gt; p < np; p += nt) I.rhs[p] = ldcg(I.yP + p);
    }
    if (!E.sync()) return false;
    if (!E.trsv(np)) return false;                 // u in yP
    // A_P u (row tiles of 32 rows, warps split the positions)
    {
      __shared__ double s_acc[NW][32];
      const int ntile = (I.m + 31) / 32;
      for (int tile = E.tm.rank; tile < ntile; tile += E.tm.size) {
        const int row = tile * 32 + lane;
        double acc = 0.0;
        if (row < I.m)
          for (int p = warp; p < np; p += NW)
            acc = fma(__ldg(I.A + (size_t)ldcg(I.order + p) * I.lda + row), ldcg(I.yP + p), acc);
        s_acc[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && row < I.m) {
          double s = 0.0;
          for (int k = 0; k < NW; ++k) s += s_acc[k][lane];
          apu[row] = s;
          if (dLdb && dLdb != apu) dLdb[row] = s;
        }
        __syncthreads();
      }
    }
    if (!E.sync()) return false;
    if (dLdA) {
      int c0, c1;
      split(I.n, E.tm.size, E.tm.rank, c0, c1);
      for (int c = c0 + warp; c < c1; c += NW) {
        const int p = ldcg(I.pos + c);
        double* out = dLdA + (size_t)c * ld_dA;
        if (p < 0 || p >= np) {
          for (int i = lane; i < I.m; i += 32) out[i] = 0.0;
        } else {
          const double up = ldcg(I.yP + p), xp = ldcg(I.xP + p);
          for (int i = lane; i < I.m; i += 32) out[i] = ldcg(I.r + i) * up - ldcg(apu + i) * xp;
        }
      }
    }
    return true;
  }
};

}  // namespace lhdm
