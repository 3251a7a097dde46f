// Nelder-Mead simplex descent on the free slots: the local search that follows the annealing in the
// paper's hybrid scheme (Section 3).  Standard coefficients (reflection 1, expansion 2, contraction
// 1/2, shrink 1/2; Lagarias, Reeds, Wright and Wright 1998), every trial point projected onto the
// box, FP64.  One team (a warp on caplet markets, a CTA on markets with swaptions) runs one
// simplex: the control flow is executed by every thread of the team on identical values (the
// objective returns the same value in every thread), slot arithmetic is spread over the threads
// t < n_param, and the team evaluates the objective cooperatively.
//
// Initial simplex: x0 and, per free slot k, x0 + step (hi_k - lo_k) e_k (downwards where it would
// leave the box).  The vertices are ordered by f with a stable insertion sort of the previous order;
// the search stops after max_iter iterations or once f_worst - f_best <= ftol |f_best|.
#pragma once
#include "market.cuh"

namespace sabr {

struct NmTeam {
  double* V;     // [(kMaxParam + 1) x kMaxParam] vertices
  double* F;     // [kMaxParam + 1]
  double* c;     // [kMaxParam] centroid
  double* xr;    // [kMaxParam] reflection
  double* xt;    // [kMaxParam] expansion / contraction trial
};

// Shared-memory bytes of one team's simplex.
__host__ __device__ constexpr uint32_t nm_team_bytes() {
  return (uint32_t)(((kMaxParam + 1) * kMaxParam + (kMaxParam + 1) + 3 * kMaxParam) * sizeof(double));
}

__device__ __forceinline__ NmTeam nm_team(double* base) {
  NmTeam s;
  s.V = base;
  s.F = s.V + (kMaxParam + 1) * kMaxParam;
  s.c = s.F + (kMaxParam + 1);
  s.xr = s.c + kMaxParam;
  s.xt = s.xr + kMaxParam;
  return s;
}

// eval(x) -> f (every thread of the team calls it, x in shared memory); sync() is the team barrier.
// t: the thread's index in the team.  x_out / f_out written by t == 0; returns the iterations run.
template <class Eval, class Sync>
__device__ int nelder_mead(const DevMarket& m, const NmTeam& s, const double* x0, int max_iter, double step,
                           double ftol, int t, Eval eval, Sync sync, double* x_out, double* f_out, int* evals_out) {
  const int P = m.n_param;
  int fi[kMaxParam];
  int nf = 0;
  for (int k = 0; k < P; ++k)
    if (m.freem[k]) fi[nf++] = k;
  const bool mine = t < P;
  const bool free_t = mine && m.freem[t] != 0;
  const double lo = mine ? m.lo[t] : 0.0, hi = mine ? m.hi[t] : 0.0;
  auto proj = [&](double v) { return fmin(fmax(v, lo), hi); };
  // initial simplex
  int vfree = -1;   // the vertex whose step moves this thread's slot
  for (int k = 0; k < nf; ++k)
    if (fi[k] == t) vfree = k + 1;
  if (mine)
    for (int k = 0; k <= nf; ++k) {
      double v = x0[t];
      if (k == vfree) {
        const double d = step * (hi - lo);
        v = x0[t] + d;
        if (v > hi) v = x0[t] - d;
        v = proj(v);
      }
      s.V[k * kMaxParam + t] = v;
    }
  sync();
  int evals = 0;
  for (int k = 0; k <= nf; ++k) {
    const double f = eval(s.V + k * kMaxParam);
    ++evals;
    if (t == 0) s.F[k] = f;
  }
  sync();
  int idx[kMaxParam + 1];
  for (int k = 0; k <= nf; ++k) idx[k] = k;
  int it = 0;
  for (;; ++it) {
    for (int i = 1; i <= nf; ++i)
      for (int j = i; j > 0 && s.F[idx[j - 1]] > s.F[idx[j]]; --j) {
        const int tmp = idx[j - 1];
        idx[j - 1] = idx[j];
        idx[j] = tmp;
      }
    const int b = idx[0], w = idx[nf], sw = idx[nf > 0 ? nf - 1 : 0];
    const double Fb = s.F[b], Fw = s.F[w], Fsw = s.F[sw];
    if (it >= max_iter || nf == 0 || !isfinite(Fb) || Fw - Fb <= ftol * fabs(Fb)) break;
    // centroid of the nf best vertices (in sorted order), the reflection
    if (mine) {
      double cv = s.V[b * kMaxParam + t];
      if (free_t) {
        double acc = 0.0;
        for (int j = 0; j < nf; ++j) acc += s.V[idx[j] * kMaxParam + t];
        cv = acc / nf;
      }
      s.c[t] = cv;
      s.xr[t] = free_t ? proj(cv + (cv - s.V[w * kMaxParam + t])) : cv;
    }
    sync();
    const double fr = eval(s.xr);
    ++evals;
    int action;   // 0: take xr, 1: try expansion, 2: outside contraction, 3: inside contraction
    if (Fb <= fr && fr < Fsw) action = 0;
    else if (fr < Fb) action = 1;
    else if (fr < Fw) action = 2;
    else action = 3;
    bool take_t = false, shrink = false;
    double ft = 0.0;
    if (action != 0) {
      if (mine) {
        const double cv = s.c[t];
        double v = cv;
        if (free_t) {
          if (action == 1) v = proj(cv + 2.0 * (s.xr[t] - cv));
          else if (action == 2) v = proj(cv + 0.5 * (s.xr[t] - cv));
          else v = proj(cv + 0.5 * (s.V[w * kMaxParam + t] - cv));
        }
        s.xt[t] = v;
      }
      sync();
      ft = eval(s.xt);
      ++evals;
      if (action == 1) take_t = ft < fr;
      else if (action == 2) { take_t = ft <= fr; shrink = !take_t; }
      else { take_t = ft < Fw; shrink = !take_t; }
    }
    if (!shrink) {
      if (mine) s.V[w * kMaxParam + t] = take_t ? s.xt[t] : s.xr[t];
      sync();
      if (t == 0) s.F[w] = take_t ? ft : fr;
      sync();
      continue;
    }
    // shrink towards the best vertex
    for (int j = 1; j <= nf; ++j) {
      const int v = idx[j];
      if (free_t) s.V[v * kMaxParam + t] = proj(s.V[b * kMaxParam + t] + 0.5 * (s.V[v * kMaxParam + t] - s.V[b * kMaxParam + t]));
      sync();
      const double f = eval(s.V + v * kMaxParam);
      ++evals;
      if (t == 0) s.F[v] = f;
      sync();
    }
  }
  const int b = idx[0];
  if (mine) x_out[t] = s.V[b * kMaxParam + t];
  if (t == 0) {
    *f_out = s.F[b];
    if (evals_out) *evals_out = evals;
  }
  sync();
  return it;
}

}  // namespace sabr
