// ok_fem.cu -- matrix-free P1 operators of the Ohta--Kawasaki system.
//
// Residual F and Jacobian J of the theta-scheme (Sec. 2, eqns oka/okb/newton),
// assembled vertex by vertex on the uniform simplex grids described in
// ok_internal.cuh.  M and K use per-class stencil tables; the variable (2,1)
// block C = -eps^2 K - M_E(u_k) is assembled once per Newton step into a
// symmetric per-vertex coefficient store (self + the NPOS positive offsets).
//
// Exact integrals on a simplex T with P1 values u_0..u_d and barycentrics
// lambda (Dirichlet moments  int_T prod lambda^k = d! |T| prod k! / (d+sum k)!):
//   int_T u_h lambda_a             = |T| d!/(d+2)! (p1 + u_a)
//   int_T u_h^3 lambda_a           = |T| d!/(d+4)! (p1^3 + 3 p1 p2 + 2 p3
//                                      + 3 u_a (p1^2 + p2) + 6 u_a^2 p1 + 6 u_a^3)
//   int_T u_h^2 lambda_a lambda_b  = |T| d!/(d+4)! (1 + delta_ab)
//                                      (p1^2 + p2 + 2 p1 (u_a + u_b) + 2 (u_a^2 + u_a u_b + u_b^2))
// with p_k = sum_c u_c^k over the simplex's vertices.  (Each follows from
// expanding prod k! as the number of label-preserving permutations of the
// integrand's factors.)  With s_k = sum of u_c^k over the vertices other than
// a (so p_k = u_a^k + s_k) the first two become
//   p1^3 + 3 p1 p2 + 2 p3 + ... = 24 a^3 + 18 a^2 s1 + 6 a (s1^2 + s2) + (s1^3 + 3 s1 s2 + 2 s3),
//   (a = b):  p1^2 + p2 + 4 p1 a + 6 a^2 = 12 a^2 + 6 a s1 + s1^2 + s2,
//   (a != b): p1^2 + p2 + 2 p1 (a + b) + 2 (a^2 + a b + b^2)
//             = 6 m^2 - 4 a b + 4 m r1 + r1^2 + r2,   m = a + b,
// r_k the power sums over the vertices other than a and b.  These are linear
// in the per-simplex sums (s1, s1^2 + s2, s1^3 + 3 s1 s2 + 2 s3, r1, r1^2 + r2),
// so a vertex sums those over its incident simplices and evaluates the
// polynomial in a once: about half the float64 operations of evaluating each
// simplex's integral separately (float64 is the bound of these kernels).
#include "ok_internal.cuh"
#include "ok_kernels.h"

namespace okg {

// ---------------------------------------------------------------------------
// host: reference class tables of M (h = 1) and K (h = 1)
// ---------------------------------------------------------------------------
template <int D>
static void reference_tables_d(double* WM, double* WK) {
  using Tp = Topo<D>;
  const double vol = 1.0 / Tp::FACT;                       // |T| of a unit simplex
  const double mcoef = vol / ((D + 1) * (D + 2));          // int lambda_a lambda_b, a != b
  for (int cls = 0; cls < Tp::NCLASS; ++cls) {
    int c[3] = {cls % 3, (cls / 3) % 3, cls / 9};
    if (D == 2) c[2] = 1;
    double* wm = WM + cls * Tp::NOFF;
    double* wk = WK + cls * Tp::NOFF;
    for (int o = 0; o < Tp::NOFF; ++o) wm[o] = wk[o] = 0.0;
    for (int i = 0; i < Tp::NINC; ++i) {
      bool ok = true;
      for (int a = 0; a < D; ++a) {
        bool neg = (inc_corner(D, i) >> a) & 1;
        ok = ok && (neg ? c[a] != 0 : c[a] != 2);
      }
      if (!ok) continue;
      int k = inc_pos(D, i);
      for (int t = 0; t <= D; ++t) {
        int o = inc_off(D, i, t);
        wm[o] += mcoef * (t == k ? 2.0 : 1.0);
        wk[o] += vol * path_lap(D, k, t);
      }
    }
  }
}

void reference_tables(int dim, double* WM, double* WK) {
  if (dim == 2) reference_tables_d<2>(WM, WK);
  else reference_tables_d<3>(WM, WK);
}

// Copy the M and K class tables into shared memory (one load per block
// instead of one per vertex and weight); call before any early return.
template <int D>
__device__ __forceinline__ void stage_tables(double* sWM, double* sWK, const double* __restrict__ WM,
                                             const double* __restrict__ WK) {
  constexpr int NT = Topo<D>::NCLASS * Topo<D>::NOFF;
  for (int i = threadIdx.x; i < NT; i += blockDim.x) {
    sWM[i] = WM[i];
    sWK[i] = WK[i];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// per-vertex simplex sums shared by N(u) and M_E(u)
// ---------------------------------------------------------------------------
template <int D> struct SimplexSums {
  double n;        // incident simplices inside the domain
  double A;        // sum s1
  double B;        // sum (s1^2 + s2)
  double C;        // sum (s1^3 + 3 s1 s2 + 2 s3)
};

// sq[o], cu[o]: squares and cubes of the neighbour values (o >= 1)
template <int D, bool CUBES>
__device__ __forceinline__ SimplexSums<D> simplex_sums(const Vtx<D>& v, const double (&us)[Topo<D>::NOFF],
                                                       const double (&sq)[Topo<D>::NOFF],
                                                       const double (&cu)[Topo<D>::NOFF]) {
  using Tp = Topo<D>;
  SimplexSums<D> z{0.0, 0.0, 0.0, 0.0};
  int n = 0;
  static_for<0, Tp::NINC>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (inc_valid<D, i>(v.c)) {
      constexpr int k = inc_pos(D, i);
      double s1 = 0.0, s2 = 0.0, s3 = 0.0;
      static_for<0, D + 1>([&](auto Tt) {
        constexpr int t = decltype(Tt)::value;
        if constexpr (t != k) {
          constexpr int o = inc_off(D, i, t);
          s1 += us[o];
          s2 += sq[o];
          if constexpr (CUBES) s3 += cu[o];
        }
      });
      ++n;
      z.A += s1;
      z.B += fma(s1, s1, s2);
      if constexpr (CUBES) z.C += fma(s1, fma(s1, s1, 3.0 * s2), 2.0 * s3);
    }
  });
  z.n = (double)n;
  return z;
}

// N(u)_v / (|T| d!): sum over the incident simplices of
//   a4 int u^3 lambda_v - a2 int u lambda_v  (a4, a2 the moment factors)
template <int D>
__device__ __forceinline__ double nonlinear_at(const Vtx<D>& v, const double (&us)[Topo<D>::NOFF], double a4,
                                               double a2) {
  using Tp = Topo<D>;
  double sq[Tp::NOFF], cu[Tp::NOFF];
#pragma unroll
  for (int o = 1; o < Tp::NOFF; ++o) {
    sq[o] = us[o] * us[o];
    cu[o] = sq[o] * us[o];
  }
  sq[0] = cu[0] = 0.0;
  const SimplexSums<D> z = simplex_sums<D, true>(v, us, sq, cu);
  const double a = us[0];
  const double t3 = fma(fma(fma(24.0 * z.n, a, 18.0 * z.A), a, 6.0 * z.B), a, z.C);
  const double lin = fma(2.0 * z.n, a, z.A);      // sum of (p1 + u_a)
  return a4 * t3 - a2 * lin;
}

// ---- 2D interior vertices: all six triangles, each neighbour in two ----------
// The triangles at a vertex pair its neighbours (offsets 1 +x, 2 -x, 3 +y,
// 4 -y, 5 +xy, 6 -xy) as (1,5) (3,5) (3,2) (2,6) (6,4) (4,1).  With the
// neighbour sums S_k = sum u_o^k, E = sum_T b c and F = sum_T b c (b + c), the
// simplex sums above are n = 6, A = 2 S1, B = 4 S2 + 2 E and, since per
// triangle s1^3 + 3 s1 s2 + 2 s3 = 6 s1 s2 for two other vertices,
// C = 6 (2 S3 + F).
__host__ __device__ constexpr int pair_b(int t) { return t == 0 ? 1 : t == 1 ? 3 : t == 2 ? 3 : t == 3 ? 2 : t == 4 ? 6 : 4; }
__host__ __device__ constexpr int pair_c(int t) { return t == 0 ? 5 : t == 1 ? 5 : t == 2 ? 2 : t == 3 ? 6 : t == 4 ? 4 : 1; }
__device__ __forceinline__ double nonlinear_interior2(const double (&us)[Topo<2>::NOFF], double a4, double a2) {
  const double a = us[0];
  double S1 = 0.0, S2 = 0.0, S3 = 0.0, E = 0.0, F = 0.0;
#pragma unroll
  for (int o = 1; o < Topo<2>::NOFF; ++o) {
    const double sq = us[o] * us[o];
    S1 += us[o];
    S2 += sq;
    S3 = fma(sq, us[o], S3);
  }
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const double bb = us[pair_b(t)], cc = us[pair_c(t)];
    const double p = bb * cc;
    E += p;
    F = fma(p, bb + cc, F);
  }
  const double t3 = fma(fma(fma(144.0, a, 36.0 * S1), a, fma(24.0, S2, 12.0 * E)), a, fma(12.0, S3, 6.0 * F));
  const double lin = fma(12.0, a, 2.0 * S1);
  return a4 * t3 - a2 * lin;
}

// path-Laplacian sums of K at an interior vertex (compile time): the diagonal
// (q = -1) and the positive offset 2q+1
__host__ __device__ constexpr int klap_interior(int D, int q) {
  int s = 0;
  for (int i = 0; i < (D == 2 ? Topo<2>::NINC : Topo<3>::NINC); ++i)
    for (int t = 0; t <= D; ++t) {
      const int o = inc_off(D, i, t);
      if ((q < 0 && t == inc_pos(D, i)) || (q >= 0 && t != inc_pos(D, i) && o == 2 * q + 1))
        s += path_lap(D, inc_pos(D, i), t);
    }
  return s;
}

// ---------------------------------------------------------------------------
// residual  f = -F(u, w)
// ---------------------------------------------------------------------------
// F1 = M g1 + K g2 with g1 = a11 u - bn u_n - dt sigma m,
//                      g2 = dt theta w + dt (1-theta) w_n,
//   a11 = 1 + dt theta sigma, bn = 1 - dt (1-theta) sigma;
// F2 = M w - eps^2 K u - N(u).
template <int D>
__global__ void __launch_bounds__(128) k_residual(Geom g, const double* __restrict__ WM,
                                                  const double* __restrict__ WK, ResidualCoefs rc,
                                                  const double* __restrict__ un, const double* __restrict__ wn,
                                                  const double* __restrict__ u, const double* __restrict__ w,
                                                  double* __restrict__ f) {
  pdl_launch_dependents();
  using Tp = Topo<D>;
  __shared__ double sWM[Tp::NCLASS * Tp::NOFF], sWK[Tp::NCLASS * Tp::NOFF];
  stage_tables<D>(sWM, sWK, WM, WK);
  pdl_wait();
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  double us[Tp::NOFF], ws[Tp::NOFF], uns[Tp::NOFF], wns[Tp::NAX];
  static_for<0, Tp::NOFF>([&](auto O) {
    constexpr int o = decltype(O)::value;
    const bool ok = nb_valid<D, o>(v.c);
    const long long j = v.idx + (ok ? nb_delta<D, o>(g) : 0);
    const double uu = u[j], ww = w[j], uun = un[j];
    us[o] = ok ? uu : 0.0;
    ws[o] = ok ? ww : 0.0;
    uns[o] = ok ? uun : 0.0;
    if constexpr (o < Tp::NAX) wns[o] = ok ? wn[j] : 0.0;
  });
  const double hd = rc.hd, hk = rc.hk;
  if constexpr (D == 2) {
    if (v.cls == 4) {            // interior: M (a11 u - bn un - dsm) = a11 M u - bn M un - dsm M 1
      const double F1 = hd * (rc.a11 * dot_w<D, Tp::NOFF>(sWM, 4, us) - rc.bn * dot_w<D, Tp::NOFF>(sWM, 4, uns) -
                              rc.dsm * rc.msum4) +
                        hk * (rc.dth * dot_w<D, Tp::NAX>(sWK, 4, ws) + rc.dth1 * dot_w<D, Tp::NAX>(sWK, 4, wns));
      double F2 = hd * dot_w<D, Tp::NOFF>(sWM, 4, ws) - rc.eps2 * hk * dot_w<D, Tp::NAX>(sWK, 4, us);
      F2 -= rc.vol * nonlinear_interior2(us, rc.a4, rc.a2);
      f[v.idx] = -F1;
      f[v.idx + g.nv] = -F2;
      return;
    }
  }
  double g1[Tp::NOFF], g2[Tp::NAX];
  static_for<0, Tp::NOFF>([&](auto O) {
    constexpr int o = decltype(O)::value;
    const bool ok = nb_valid<D, o>(v.c);
    g1[o] = ok ? (rc.a11 * us[o] - rc.bn * uns[o] - rc.dsm) : 0.0;
    if constexpr (o < Tp::NAX) g2[o] = ok ? (rc.dth * ws[o] + rc.dth1 * wns[o]) : 0.0;
  });
  double F1 = hd * dot_w<D, Tp::NOFF>(sWM, v.cls, g1) + hk * dot_w<D, Tp::NAX>(sWK, v.cls, g2);
  double F2 = hd * dot_w<D, Tp::NOFF>(sWM, v.cls, ws) - rc.eps2 * hk * dot_w<D, Tp::NAX>(sWK, v.cls, us);
  // N(u)_v: sums over the incident simplices
  F2 -= rc.vol * nonlinear_at<D>(v, us, rc.a4, rc.a2);
  f[v.idx] = -F1;
  f[v.idx + g.nv] = -F2;
}

// rhs of the w0 projection: eps^2 K u0 + N(u0)
template <int D>
__global__ void __launch_bounds__(128) k_initw_rhs(Geom g, const double* __restrict__ WK, ResidualCoefs rc,
                                                   const double* __restrict__ u, double* __restrict__ out) {
  pdl_entry();
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  double us[Tp::NOFF];
  load_nb<D>(u, g, v, us);
  double acc = rc.eps2 * rc.hk * dot_w<D, Tp::NAX>(WK, v.cls, us);
  out[v.idx] = acc + rc.vol * nonlinear_at<D>(v, us, rc.a4, rc.a2);
}

// ---------------------------------------------------------------------------
// Local terms of the Ohta--Kawasaki energy (Sec. 1) per vertex v:
//   e[v]       = eps^2/2 u_v (K u)_v                       (sums to eps^2/2 u^T K u)
//   e[N_v + v] = 1/4 sum over the simplices T at v of int_T (1 - u_h^2)^2 / (d+1)
// (each simplex is shared by its d+1 vertices, so the second sums to
// 1/4 int (1 - u_h^2)^2).  On T with vertex values u_0..u_d and power sums
// p_k = sum u_c^k (Dirichlet moments, as above):
//   int_T u_h^2 = |T| d!/(d+2)! (p1^2 + p2),
//   int_T u_h^4 = |T| d!/(d+4)! (p1^4 + 6 p1^2 p2 + 3 p2^2 + 8 p1 p3 + 6 p4)
// (the complete homogeneous symmetric polynomials h2 and h4 times 2! and 4!).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(128) k_energy_local(Geom g, const double* __restrict__ WK, ResidualCoefs rc,
                                                      const double* __restrict__ u, double* __restrict__ e) {
  pdl_entry();
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  double us[Tp::NOFF];
  load_nb<D>(u, g, v, us);
  const double ku = rc.hk * dot_w<D, Tp::NAX>(WK, v.cls, us);
  double well = 0.0;
  static_for<0, Tp::NINC>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (inc_valid<D, i>(v.c)) {
      double p1 = 0.0, p2 = 0.0, p3 = 0.0, p4 = 0.0;
      static_for<0, D + 1>([&](auto Tt) {
        constexpr int o = inc_off(D, i, decltype(Tt)::value);
        const double x = us[o], x2 = x * x;
        p1 += x;
        p2 += x2;
        p3 = fma(x2, x, p3);
        p4 = fma(x2, x2, p4);
      });
      const double q2 = fma(p1, p1, p2);
      const double q4 = fma(p1 * p1, fma(p1, p1, 6.0 * p2), fma(3.0 * p2, p2, fma(8.0 * p1, p3, 6.0 * p4)));
      well += fma(-2.0 * rc.a2, q2, fma(rc.a4, q4, 1.0));
    }
  });
  e[v.idx] = 0.5 * rc.eps2 * us[0] * ku;
  e[g.nv + v.idx] = 0.25 * rc.vol * well / (D + 1);
}

// ---------------------------------------------------------------------------
// C = -eps^2 K - M_E(u) coefficients, symmetric storage:
//   coef[0][v]   = C(v, v)
//   coef[1+p][v] = C(v, v + pos_p)       (p = 0..NPOS-1)
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(128) k_assemble_c(Geom g, ResidualCoefs rc, const double* __restrict__ u,
                                                    double* __restrict__ coef, float* __restrict__ coef32) {
  pdl_entry();
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  double us[Tp::NOFF];
  load_nb<D>(u, g, v, us);
  double sq[Tp::NOFF];
#pragma unroll
  for (int o = 0; o < Tp::NOFF; ++o) sq[o] = us[o] * us[o];
  const double kscale = rc.eps2 * rc.hk * (1.0 / Tp::FACT);   // eps^2 h^(d-2) / d!
  const double a = us[0];
  if constexpr (D == 2) {
    if (v.cls == 4) {            // interior: six triangles, each edge in two
      double S1 = 0.0, S2 = 0.0, E = 0.0;
#pragma unroll
      for (int o = 1; o < Tp::NOFF; ++o) {
        S1 += us[o];
        S2 += sq[o];
      }
#pragma unroll
      for (int t = 0; t < 6; ++t) E = fma(us[pair_b(t)], us[pair_c(t)], E);
      // sum over the triangles of p1^2 + p2 + 4 p1 a + 6 a^2 = 12 n a^2 + 6 a A + B
      const double Paa = fma(fma(72.0, a, 12.0 * S1), a, fma(4.0, S2, 2.0 * E));
      constexpr int KL0 = klap_interior(2, -1);
      const double diag = -kscale * KL0 - rc.vol * 2.0 * (3.0 * rc.a4 * Paa - rc.a2 * 6.0);
      coef[v.idx] = diag;
      coef32[v.idx] = (float)diag;
      // edge (v, v + pos_q) lies in two triangles whose third vertices are c1, c2
      static_for<0, Tp::NPOS>([&](auto Q) {
        constexpr int q = decltype(Q)::value;
        constexpr int t1 = q == 0 ? 5 : (q == 1 ? 5 : 1), t2 = q == 0 ? 4 : (q == 1 ? 2 : 3);
        const double b = us[2 * q + 1], c1 = us[t1], c2 = us[t2];
        const double m = a + b;
        const double R1 = c1 + c2, R2 = 2.0 * (sq[t1] + sq[t2]);
        const double P = fma(2.0, fma(6.0 * m, m, -4.0 * a * b), fma(4.0 * m, R1, R2));
        constexpr int KLQ = klap_interior(2, q);
        const double c = -kscale * KLQ - rc.vol * (3.0 * rc.a4 * P - rc.a2 * 2.0);
        coef[(1 + q) * g.nv + v.idx] = c;
        coef32[(1 + q) * g.nv + v.idx] = (float)c;
      });
      return;
    }
  }
  // per positive offset p: simplices holding the edge, sum r1, sum (r1^2 + r2),
  // and the summed path-Laplacian entries of K
  double R1[Tp::NPOS], R2[Tp::NPOS];
  int ne[Tp::NPOS], kl[Tp::NPOS + 1];
#pragma unroll
  for (int q = 0; q < Tp::NPOS; ++q) R1[q] = R2[q] = 0.0, ne[q] = 0;
#pragma unroll
  for (int q = 0; q <= Tp::NPOS; ++q) kl[q] = 0;
  int n = 0;
  double A = 0.0, B = 0.0;
  static_for<0, Tp::NINC>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (inc_valid<D, i>(v.c)) {
      constexpr int k = inc_pos(D, i);
      double s1 = 0.0, s2 = 0.0;
      static_for<0, D + 1>([&](auto Tt) {
        constexpr int t = decltype(Tt)::value;
        if constexpr (t != k) {
          constexpr int o = inc_off(D, i, t);
          s1 += us[o];
          s2 += sq[o];
        }
      });
      ++n;
      A += s1;
      B += fma(s1, s1, s2);
      kl[0] += path_lap(D, k, k);
      static_for<0, D + 1>([&](auto Tt) {
        constexpr int t = decltype(Tt)::value;
        constexpr int o = inc_off(D, i, t);
        if constexpr (t != k && (o & 1)) {          // a positive offset: C(v, v + pos) is stored here
          constexpr int q = (o - 1) / 2;
          const double r1 = s1 - us[o];
          const double r2 = s2 - sq[o];
          R1[q] += r1;
          R2[q] += fma(r1, r1, r2);
          ne[q] += 1;
          kl[q + 1] += path_lap(D, k, t);
        }
      });
    }
  });
  // M_E entries: 3 int u^2 l_a l_b - int l_a l_b  (times vol, 2x on the diagonal)
  const double nd = (double)n;
  const double Paa = fma(fma(12.0 * nd, a, 6.0 * A), a, B);
  const double diag = -kscale * kl[0] - rc.vol * 2.0 * (3.0 * rc.a4 * Paa - rc.a2 * nd);
  coef[v.idx] = diag;
  coef32[v.idx] = (float)diag;
#pragma unroll
  for (int q = 0; q < Tp::NPOS; ++q) {
    const double b = us[2 * q + 1];
    const double m = a + b, nq = (double)ne[q];
    const double P = fma(nq, fma(6.0 * m, m, -4.0 * a * b), fma(4.0 * m, R1[q], R2[q]));
    const double c = -kscale * kl[q + 1] - rc.vol * (3.0 * rc.a4 * P - rc.a2 * nq);
    coef[(1 + q) * g.nv + v.idx] = c;
    coef32[(1 + q) * g.nv + v.idx] = (float)c;
  }
}

// sum over the symmetric store: (C y)_v
template <int D, typename T, typename TY>
__device__ __forceinline__ T capply_at(const Geom& g, const Vtx<D>& v, const T* __restrict__ coef,
                                       const TY* __restrict__ y, T yscale) {
  using Tp = Topo<D>;
  T acc = coef[v.idx] * (T)y[v.idx] * yscale;
  static_for<0, Tp::NPOS>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int op = 2 * p + 1, om = 2 * p + 2;
    if (nb_valid<D, op>(v.c)) {
      long long j = v.idx + nb_delta<D, op>(g);
      acc = fma(coef[(1 + p) * g.nv + v.idx], (T)y[j] * yscale, acc);
    }
    if (nb_valid<D, om>(v.c)) {
      long long j = v.idx + nb_delta<D, om>(g);
      acc = fma(coef[(1 + p) * g.nv + j], (T)y[j] * yscale, acc);
    }
  });
  return acc;
}

// The same sum from neighbour values already loaded (ys[o] = y at offset o,
// converted once): no second load and no second float->double conversion.
template <int D, typename T>
__device__ __forceinline__ T capply_from(const Geom& g, const Vtx<D>& v, const T* __restrict__ coef,
                                         const T (&ys)[Topo<D>::NOFF]) {
  using Tp = Topo<D>;
  T acc = coef[v.idx] * ys[0];
  static_for<0, Tp::NPOS>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int op = 2 * p + 1, om = 2 * p + 2;
    if (nb_valid<D, op>(v.c)) acc = fma(coef[(1 + p) * g.nv + v.idx], ys[op], acc);
    if (nb_valid<D, om>(v.c)) acc = fma(coef[(1 + p) * g.nv + v.idx + nb_delta<D, om>(g)], ys[om], acc);
  });
  return acc;
}


template <int D, typename TX>
__device__ __forceinline__ void load_nb_d(const TX* __restrict__ x, const Geom& g, const Vtx<D>& v,
                                          double (&out)[Topo<D>::NOFF]) {
  if constexpr (std::is_same<TX, float>::value) {
    static_for<0, Topo<D>::NOFF>([&](auto O) {
      constexpr int o = decltype(O)::value;
      out[o] = nb_valid<D, o>(v.c) ? f2d_exact(x[v.idx + nb_delta<D, o>(g)]) : 0.0;
    });
  } else if constexpr (std::is_same<TX, __half>::value) {   // half -> float (exact) -> double
    static_for<0, Topo<D>::NOFF>([&](auto O) {
      constexpr int o = decltype(O)::value;
      out[o] = nb_valid<D, o>(v.c) ? f2d_exact(__half2float(x[v.idx + nb_delta<D, o>(g)])) : 0.0;
    });
  } else {
    load_nb<D>(x, g, v, out);
  }
}

// ---------------------------------------------------------------------------
// y = alpha J z + beta y0, J = [a11 M, dth K; C, M]  (eqn newton)
// ---------------------------------------------------------------------------
template <int D, typename TZ>
__device__ __forceinline__ void apply_j_body(const Geom& g, int kz, const double* __restrict__ WM,
                                             const double* __restrict__ WK, const JCoefs& jc,
                                             const double* __restrict__ coef, const TZ* __restrict__ z,
                                             double* __restrict__ y, const double* __restrict__ y0) {
  using Tp = Topo<D>;
  __shared__ double sWM[Tp::NCLASS * Tp::NOFF], sWK[Tp::NCLASS * Tp::NOFF];
  stage_tables<D>(sWM, sWK, WM, WK);
  pdl_wait();
  Vtx<D> v;
  if (!vertex_of_thread_at<D>(g, kz, v)) return;
  double z1[Tp::NOFF], z2[Tp::NOFF];
  load_nb_d<D, TZ>(z, g, v, z1);
  load_nb_d<D, TZ>(z + g.nv, g, v, z2);
  // every product that feeds a sum is an explicit fma, so each kernel that
  // inlines this body (one problem or a batch) rounds the same way
  const double mz1 = dot_w<D, Tp::NOFF>(sWM, v.cls, z1);
  const double kz2 = dot_w<D, Tp::NAX>(sWK, v.cls, z2);
  const double mz2 = dot_w<D, Tp::NOFF>(sWM, v.cls, z2);
  const double cz1 = capply_from<D, double>(g, v, coef, z1);
  double y1 = fma(jc.a11hd, mz1, jc.dthhk * kz2);
  double y2 = fma(jc.hd, mz2, cz1);
  if (y0) {
    y1 = fma(jc.beta, y0[v.idx], jc.alpha * y1);
    y2 = fma(jc.beta, y0[v.idx + g.nv], jc.alpha * y2);
  }
  y[v.idx] = y1;
  y[v.idx + g.nv] = y2;
}
template <int D, typename TZ>
__global__ void __launch_bounds__(128) k_apply_j(Geom g, const double* __restrict__ WM,
                                                 const double* __restrict__ WK, JCoefs jc,
                                                 const double* __restrict__ coef, const TZ* __restrict__ z,
                                                 double* __restrict__ y, const double* __restrict__ y0) {
  pdl_launch_dependents();
  apply_j_body<D, TZ>(g, D == 3 ? (int)blockIdx.z : 0, WM, WK, jc, coef, z, y, y0);
}
template <int D, typename TZ>
__global__ void __launch_bounds__(128) k_apply_j_b(Batch<ApplyJItem<TZ>> B, Geom g, const double* __restrict__ WM,
                                                   const double* __restrict__ WK) {
  pdl_launch_dependents();
  const ApplyJItem<TZ>& a = B.a[batch_problem<D>(g)];
  apply_j_body<D, TZ>(g, batch_plane<D>(g), WM, WK, a.jc, a.coef, a.z, a.y, (const double*)nullptr);
}

// ---------------------------------------------------------------------------
// preconditioner C-step:  t = s * v2 - C (ys * y1)     (eqn prec: r2 - C A^{-1} r1)
// ---------------------------------------------------------------------------
template <int D, typename T, typename TV>
__global__ void __launch_bounds__(128) k_cstep(Geom g, const T* __restrict__ coef, const TV* __restrict__ v2,
                                               T vscale, const T* __restrict__ y1, T yscale, T* __restrict__ t) {
  pdl_entry();
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T cy = capply_at<D, T>(g, v, coef, y1, yscale);
  t[v.idx] = fma((T)v2[v.idx], vscale, -cy);
}
template <int D, typename T, typename TV>
__global__ void __launch_bounds__(128) k_cstep_b(Batch<CStepItem<T, TV>> B, Geom g) {
  pdl_entry();
  const CStepItem<T, TV>& a = B.a[batch_problem<D>(g)];
  Vtx<D> v;
  if (!vertex_of_thread_at<D>(g, batch_plane<D>(g), v)) return;
  T cy = capply_at<D, T>(g, v, a.coef, a.y1, a.yscale);
  a.t[v.idx] = fma((T)a.v2[v.idx], a.vscale, -cy);
}

// Richardson residual for k_R = 2:  out = t - (M y - C a)   (S y = M y - C A~^{-1} B y)
template <int D, typename T>
__global__ void __launch_bounds__(128) k_schur_resid(Geom g, const T* __restrict__ WM, T hd, const T* __restrict__ coef,
                                                     const T* __restrict__ t, const T* __restrict__ y,
                                                     const T* __restrict__ a, T ascale, T* __restrict__ out) {
  pdl_entry();
  using Tp = Topo<D>;
  Vtx<D> v;
  if (!vertex_of_thread<D>(g, v)) return;
  T ys[Tp::NOFF];
  load_nb<D>(y, g, v, ys);
  T my = hd * dot_w<D, Tp::NOFF>(WM, v.cls, ys);
  T ca = capply_at<D, T>(g, v, coef, a, ascale);
  out[v.idx] = t[v.idx] - my + ca;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline dim3 grid_of(int dim, const Geom& g, int bx) {
  return dim3((unsigned)(((long long)g.n1 * g.n1 + bx - 1) / bx), 1, dim == 3 ? g.n1 : 1);
}

void launch_residual(int dim, const Geom& g, const double* WM, const double* WK, const ResidualCoefs& rc,
                     const double* un, const double* wn, const double* u, const double* w, double* f,
                     cudaStream_t s) {
  dim3 grd = grid_of(dim, g, 128);
  if (dim == 2) launch_k(k_residual<2>, grd, 128, 0, s, g, WM, WK, rc, un, wn, u, w, f);
  else launch_k(k_residual<3>, grd, 128, 0, s, g, WM, WK, rc, un, wn, u, w, f);
}

void launch_initw_rhs(int dim, const Geom& g, const double* WK, const ResidualCoefs& rc, const double* u,
                      double* out, cudaStream_t s) {
  dim3 grd = grid_of(dim, g, 128);
  if (dim == 2) launch_k(k_initw_rhs<2>, grd, 128, 0, s, g, WK, rc, u, out);
  else launch_k(k_initw_rhs<3>, grd, 128, 0, s, g, WK, rc, u, out);
}

void launch_energy_local(int dim, const Geom& g, const double* WK, const ResidualCoefs& rc, const double* u,
                         double* e, cudaStream_t s) {
  dim3 grd = grid_of(dim, g, 128);
  if (dim == 2) launch_k(k_energy_local<2>, grd, 128, 0, s, g, WK, rc, u, e);
  else launch_k(k_energy_local<3>, grd, 128, 0, s, g, WK, rc, u, e);
}

void launch_assemble_c(int dim, const Geom& g, const ResidualCoefs& rc, const double* u, double* coef,
                       float* coef32, cudaStream_t s) {
  dim3 grd = grid_of(dim, g, 128);
  if (dim == 2) launch_k(k_assemble_c<2>, grd, 128, 0, s, g, rc, u, coef, coef32);
  else launch_k(k_assemble_c<3>, grd, 128, 0, s, g, rc, u, coef, coef32);
}

template <typename TZ>
void launch_apply_j(int dim, const Geom& g, const double* WM, const double* WK, const JCoefs& jc,
                    const double* coef, const TZ* z, double* y, const double* y0, cudaStream_t s) {
  dim3 grd = grid_of(dim, g, 128);
  if (dim == 2) launch_k(k_apply_j<2, TZ>, grd, 128, 0, s, g, WM, WK, jc, coef, z, y, y0);
  else launch_k(k_apply_j<3, TZ>, grd, 128, 0, s, g, WM, WK, jc, coef, z, y, y0);
}
template <typename TZ>
void launch_apply_j_b(int dim, const Geom& g, const double* WM, const double* WK, const ApplyJItem<TZ>* items,
                      int count, cudaStream_t s) {
  Batch<ApplyJItem<TZ>> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  dim3 grd = grid_of(dim, g, 128);
  grd.z *= count;
  if (dim == 2) launch_k(k_apply_j_b<2, TZ>, grd, 128, 0, s, B, g, WM, WK);
  else launch_k(k_apply_j_b<3, TZ>, grd, 128, 0, s, B, g, WM, WK);
}
template void launch_apply_j_b<double>(int, const Geom&, const double*, const double*, const ApplyJItem<double>*,
                                       int, cudaStream_t);
template void launch_apply_j_b<float>(int, const Geom&, const double*, const double*, const ApplyJItem<float>*,
                                      int, cudaStream_t);
template void launch_apply_j_b<__half>(int, const Geom&, const double*, const double*, const ApplyJItem<__half>*,
                                       int, cudaStream_t);
template <typename T, typename TV>
void launch_cstep_b(int dim, const Geom& g, const CStepItem<T, TV>* items, int count, cudaStream_t s) {
  Batch<CStepItem<T, TV>> B;
  for (int i = 0; i < count; ++i) B.a[i] = items[i];
  dim3 grd = grid_of(dim, g, 128);
  grd.z *= count;
  if (dim == 2) launch_k(k_cstep_b<2, T, TV>, grd, 128, 0, s, B, g);
  else launch_k(k_cstep_b<3, T, TV>, grd, 128, 0, s, B, g);
}
template void launch_cstep_b<double, double>(int, const Geom&, const CStepItem<double, double>*, int, cudaStream_t);
template void launch_cstep_b<float, double>(int, const Geom&, const CStepItem<float, double>*, int, cudaStream_t);
template void launch_apply_j<double>(int, const Geom&, const double*, const double*, const JCoefs&,
                                     const double*, const double*, double*, const double*, cudaStream_t);
template void launch_apply_j<float>(int, const Geom&, const double*, const double*, const JCoefs&,
                                    const double*, const float*, double*, const double*, cudaStream_t);
template void launch_apply_j<__half>(int, const Geom&, const double*, const double*, const JCoefs&,
                                     const double*, const __half*, double*, const double*, cudaStream_t);

template <typename T, typename TV>
void launch_cstep(int dim, const Geom& g, const T* coef, const TV* v2, T vscale, const T* y1, T yscale, T* t,
                  cudaStream_t s) {
  dim3 grd = grid_of(dim, g, 128);
  if (dim == 2) launch_k(k_cstep<2, T, TV>, grd, 128, 0, s, g, coef, v2, vscale, y1, yscale, t);
  else launch_k(k_cstep<3, T, TV>, grd, 128, 0, s, g, coef, v2, vscale, y1, yscale, t);
}
template void launch_cstep<double, double>(int, const Geom&, const double*, const double*, double, const double*,
                                           double, double*, cudaStream_t);
template void launch_cstep<float, double>(int, const Geom&, const float*, const double*, float, const float*, float,
                                          float*, cudaStream_t);

template <typename T>
void launch_schur_resid(int dim, const Geom& g, const T* WM, T hd, const T* coef, const T* t, const T* y,
                        const T* a, T ascale, T* out, cudaStream_t s) {
  dim3 grd = grid_of(dim, g, 128);
  if (dim == 2) launch_k(k_schur_resid<2, T>, grd, 128, 0, s, g, WM, hd, coef, t, y, a, ascale, out);
  else launch_k(k_schur_resid<3, T>, grd, 128, 0, s, g, WM, hd, coef, t, y, a, ascale, out);
}
template void launch_schur_resid<double>(int, const Geom&, const double*, double, const double*, const double*,
                                         const double*, const double*, double, double*, cudaStream_t);
template void launch_schur_resid<float>(int, const Geom&, const float*, float, const float*, const float*,
                                        const float*, const float*, float, float*, cudaStream_t);

}  // namespace okg
