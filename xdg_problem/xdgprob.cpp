// Generator of the agglomerated XDG-SIP system (input of the multigrid solve).
//
// Kummer, Smuda, Weber, arXiv 2003.02431. Section references are to that paper:
//   sec. 1.1  Poisson problem with a jump in mu, level set, species, interface normal
//   sec. 2    DG/XDG spaces, cut-cell mesh, jump/mean operators, SIP form (Eq. DefSIP),
//             right-hand side (Eq. SIPrhs), penalty scaling with the agglomerated cell
//   sec. 2.3  agglomeration map A_alpha (volume fraction <= alpha, same species, largest neighbour)
//   sec. 3.1  aggregation sequence on the background mesh, duplication per species,
//             level maps A'^lambda = (A^lambda)^X U A_alpha
//   sec. 3.2  basis on the bounding box of an aggregate, re-orthonormalisation S by
//             Cholesky, transfer R^{X,lambda} (Eq. XDGrestrictionMatrix), minimum background
//             cell index as representative
//
// Cut-cell quadrature follows Saye's dimension-reduction method for hyperrectangles
// (R. Saye, SIAM J. Sci. Comput. 37 (2015)), which the paper names as one of its two
// quadrature options; here it is written for the sphere/circle level sets of the
// workloads, for which every restricted function is again |x - c|^2 + kappa over the
// remaining coordinates and every root along a coordinate line has a closed form.
#include "xdgprob.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ------------------------------------------------------------------------------------------
// 1-D Gauss-Legendre rules on [0,1] (Newton iteration on the Legendre recurrence)
// ------------------------------------------------------------------------------------------
struct Rule1 {
  std::vector<double> u, w;
};

Rule1 gauss01(int n) {
  Rule1 r;
  r.u.resize(n);
  r.w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    r.u[i] = 0.5 * (1.0 - z);
    r.w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)P'^2) scaled to [0,1]
  }
  return r;
}

// Legendre polynomials P_0..P_k and derivatives at t in [-1,1]
inline void legendre(int k, double t, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (k >= 1) {
    P[1] = t;
    dP[1] = 1.0;
  }
  for (int n = 1; n < k; ++n) {
    P[n + 1] = ((2.0 * n + 1.0) * t * P[n] - n * P[n - 1]) / (n + 1.0);
    dP[n + 1] = dP[n - 1] + (2.0 * n + 1.0) * P[n];
  }
}

// ------------------------------------------------------------------------------------------
// small dense helpers (row-major n x n)
// ------------------------------------------------------------------------------------------
// Cholesky A = L L^T in place (lower triangle), returns false if not positive definite
bool cholesky(int n, double* A) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int p = 0; p < j; ++p) s -= A[j * n + p] * A[j * n + p];
    if (!(s > 0.0)) return false;
    double d = std::sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int p = 0; p < j; ++p) t -= A[i * n + p] * A[j * n + p];
      A[i * n + j] = t / d;
    }
    for (int i = 0; i < j; ++i) A[i * n + j] = 0.0;
  }
  return true;
}

// X := T * L^{-T}  (T is r x n, L lower n x n): solve X L^T = T row by row
void right_solve_LT(int r, int n, const double* L, const double* T, double* X) {
  for (int i = 0; i < r; ++i) {
    for (int j = 0; j < n; ++j) {
      double s = T[i * n + j];
      for (int p = 0; p < j; ++p) s -= X[i * n + p] * L[j * n + p];
      X[i * n + j] = s / L[j * n + j];
    }
  }
}

// Y := L^{-1} X  (X is n x c)
void left_solve_L(int n, int c, const double* L, double* X) {
  for (int col = 0; col < c; ++col) {
    for (int i = 0; i < n; ++i) {
      double s = X[i * c + col];
      for (int p = 0; p < i; ++p) s -= L[i * n + p] * X[p * c + col];
      X[i * c + col] = s / L[i * n + i];
    }
  }
}

// C = A^T B (A: r x n, B: r x m -> C: n x m), accumulate if acc
void gemm_tn(int r, int n, int m, const double* A, const double* B, double* C, bool acc) {
  if (!acc) std::fill(C, C + (size_t)n * m, 0.0);
  for (int p = 0; p < r; ++p)
    for (int i = 0; i < n; ++i) {
      double a = A[p * n + i];
      if (a == 0.0) continue;
      for (int j = 0; j < m; ++j) C[i * m + j] += a * B[p * m + j];
    }
}

// C = A B (A: n x r, B: r x m)
void gemm_nn(int n, int r, int m, const double* A, const double* B, double* C) {
  std::fill(C, C + (size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int p = 0; p < r; ++p) {
      double a = A[i * r + p];
      if (a == 0.0) continue;
      for (int j = 0; j < m; ++j) C[i * m + j] += a * B[p * m + j];
    }
}

// ------------------------------------------------------------------------------------------
// Saye-type quadrature on a hyperrectangle for functions psi = sum_{free d}(x_d-c_d)^2 + kappa
// ------------------------------------------------------------------------------------------
struct Fn {
  double kappa;
  int s;       // required sign (+1, -1) or 0 (only a break point)
  bool sing;   // the integrand of the enclosing level has a square-root branch on psi = 0
  bool ghost;  // carries a branch locus only: neither a break point nor a sign condition
};
struct QP {
  double x[3];
  double w;
};

struct Saye {
  int D;
  double c[3];
  Rule1 g;  // q-point rule on [0,1]

  // q-point rule on [t0,t1]; a square-root branch point at SL <= t0 (or SR >= t1) that lies
  // within one interval length is absorbed by t = S +- (t - S) v^2 (Gauss in v).
  void interval(double t0, double t1, double SL, double SR,
                std::vector<std::pair<double, double>>& pts) const {
    double L = t1 - t0;
    if (!(L > 0)) return;
    const int q = (int)g.u.size();
    bool nl = (t0 - SL) <= L, nr = (SR - t1) <= L;
    if (nl && nr) {
      double mid = 0.5 * (t0 + t1);
      interval(t0, mid, SL, 1e300, pts);
      interval(mid, t1, -1e300, SR, pts);
      return;
    }
    if (!nl && !nr) {
      for (int i = 0; i < q; ++i) pts.push_back({t0 + L * g.u[i], L * g.w[i]});
    } else if (nl) {  // t = SL + (t1 - SL) v^2, v in [v0, 1]
      double A = t1 - SL, v0 = std::sqrt(std::max(0.0, (t0 - SL) / A)), lv = 1.0 - v0;
      for (int i = 0; i < q; ++i) {
        double v = v0 + lv * g.u[i];
        pts.push_back({SL + A * v * v, 2.0 * A * v * lv * g.w[i]});
      }
    } else {  // t = SR - (SR - t0) v^2
      double A = SR - t0, v0 = std::sqrt(std::max(0.0, (SR - t1) / A)), lv = 1.0 - v0;
      for (int i = 0; i < q; ++i) {
        double v = v0 + lv * g.u[i];
        pts.push_back({SR - A * v * v, 2.0 * A * v * lv * g.w[i]});
      }
    }
  }

  // range of sum_{d in fr}(x_d - c_d)^2 over the box
  void sq_range(int m, const int* fr, const double* a, const double* b, double& lo,
                double& hi) const {
    lo = hi = 0.0;
    for (int i = 0; i < m; ++i) {
      int d = fr[i];
      double u = a[d] - c[d], v = b[d] - c[d];
      double uu = u * u, vv = v * v;
      hi += std::max(uu, vv);
      lo += (u <= 0.0 && v >= 0.0) ? 0.0 : std::min(uu, vv);
    }
  }

  // m free dims fr[0..m), box [a,b] (indexed by global dim), fixed coordinates in x0.
  // surf >= 0: integrate over the zero set of fns[surf] (surface measure); else volume.
  void rec(int m, const int* fr, const double* a, const double* b, const double* x0,
           std::vector<Fn> fns, int surf, std::vector<QP>& out) const {
    // 1. prune functions of uniform sign
    double rlo, rhi;
    sq_range(m, fr, a, b, rlo, rhi);
    std::vector<Fn> keep;
    int surf_k = -1;
    bool any_real = false;
    for (int i = 0; i < (int)fns.size(); ++i) {
      double lo = rlo + fns[i].kappa, hi = rhi + fns[i].kappa;
      if (fns[i].ghost) {
        keep.push_back(fns[i]);
        continue;
      }
      if (i == surf) {
        if (!(lo < 0.0 && hi > 0.0)) return;
        surf_k = (int)keep.size();
        keep.push_back(fns[i]);
        any_real = true;
        continue;
      }
      if (lo >= 0.0 || hi <= 0.0) {
        int sg = (lo >= 0.0) ? 1 : -1;
        if (fns[i].s != 0 && fns[i].s != sg) return;
        if (!fns[i].sing) continue;
        // a branch locus outside the box still shapes the integrand: keep it as a ghost
        Fn gh = fns[i];
        gh.ghost = true;
        gh.s = 0;
        keep.push_back(gh);
        continue;
      }
      keep.push_back(fns[i]);
      any_real = true;
    }
    if (!any_real) {  // tensor-product rule on the box (graded towards branch loci)
      std::vector<QP> cur(1);
      for (int d = 0; d < 3; ++d) cur[0].x[d] = x0[d];
      cur[0].w = 1.0;
      if (keep.empty() || m == 0) {
        std::vector<std::pair<double, double>> pts;
        for (int i = 0; i < m; ++i) {
          int d = fr[i];
          std::vector<QP> nxt;
          pts.clear();
          interval(a[d], b[d], -1e300, 1e300, pts);
          for (const QP& p : cur)
            for (auto& pw : pts) {
              QP r = p;
              r.x[d] = pw.first;
              r.w = p.w * pw.second;
              nxt.push_back(r);
            }
          cur.swap(nxt);
        }
        out.insert(out.end(), cur.begin(), cur.end());
        return;
      }
    }
    // 2. height direction: the gradient component 2(x_k-c_k) must keep its sign on the box
    int k = -1;
    double best = -1.0;
    for (int i = 0; i < m; ++i) {
      int d = fr[i];
      if (c[d] <= a[d] || c[d] >= b[d]) {
        double gk = std::fabs(0.5 * (a[d] + b[d]) - c[d]);
        if (gk > best) {
          best = gk;
          k = d;
        }
      }
    }
    if (k < 0) {  // the centre is inside the box: split it at the centre
      int sd[3], ns = 0;
      for (int i = 0; i < m; ++i)
        if (c[fr[i]] > a[fr[i]] && c[fr[i]] < b[fr[i]]) sd[ns++] = fr[i];
      for (int mask = 0; mask < (1 << ns); ++mask) {
        double a2[3], b2[3];
        for (int d = 0; d < 3; ++d) {
          a2[d] = a[d];
          b2[d] = b[d];
        }
        for (int j = 0; j < ns; ++j) {
          int d = sd[j];
          if (mask & (1 << j)) a2[d] = c[d];
          else b2[d] = c[d];
        }
        rec(m, fr, a2, b2, x0, keep, surf_k, out);
      }
      return;
    }
    const int sigma = (a[k] >= c[k]) ? 1 : -1;
    const double gap = std::min(std::fabs(a[k] - c[k]), std::fabs(b[k] - c[k]));
    const bool touchL = (a[k] == c[k]), touchU = (b[k] == c[k]);
    const bool near = !touchL && !touchU && gap <= (b[k] - a[k]);
    const double dL = (a[k] - c[k]) * (a[k] - c[k]), dU = (b[k] - c[k]) * (b[k] - c[k]);
    // 3. functions of the (m-1)-dimensional base problem
    std::vector<Fn> base_fns;
    auto add_fn = [&](Fn f) -> bool {
      for (Fn& e : base_fns)
        if (e.kappa == f.kappa) {
          if (e.ghost && !f.ghost) {
            e.ghost = false;
            e.s = f.s;
          } else if (!f.ghost) {
            if (e.s == 0) e.s = f.s;
            else if (f.s != 0 && f.s != e.s) return false;
          }
          e.sing = e.sing || f.sing;
          return true;
        }
      base_fns.push_back(f);
      return true;
    };
    for (int i = 0; i < (int)keep.size(); ++i) {
      const Fn& f = keep[i];
      if (f.ghost) {
        add_fn({f.kappa + dL, 0, true, true});
        add_fn({f.kappa + dU, 0, true, true});
        if (near) add_fn({f.kappa, 0, true, true});
        continue;
      }
      int sL, sU;
      if (i == surf_k) {
        sL = -sigma;
        sU = sigma;
      } else {
        sL = (f.s == sigma) ? 0 : f.s;
        sU = (f.s == -sigma) ? 0 : f.s;
      }
      if (!add_fn({f.kappa + dL, sL, f.sing || touchL, false})) return;
      if (!add_fn({f.kappa + dU, sU, f.sing || touchU, false})) return;
      // the lifted integrand has a branch where the root reaches x_k = c_k
      if (near) add_fn({f.kappa, 0, true, true});
    }
    int fr2[3], m2 = 0;
    for (int i = 0; i < m; ++i)
      if (fr[i] != k) fr2[m2++] = fr[i];
    std::vector<QP> base;
    rec(m2, fr2, a, b, x0, base_fns, -1, base);
    // 4. lift along x_k
    std::vector<std::pair<double, bool>> roots;
    std::vector<double> spts;
    std::vector<std::pair<double, double>> pts;
    for (const QP& bp : base) {
      double r0 = 0.0;
      for (int i = 0; i < m2; ++i) {
        double t = bp.x[fr2[i]] - c[fr2[i]];
        r0 += t * t;
      }
      if (surf_k >= 0) {
        double rho = r0 + keep[surf_k].kappa;
        if (!(rho < 0.0)) continue;
        double t = c[k] + sigma * std::sqrt(-rho);
        if (t < a[k] || t > b[k]) continue;
        bool ok = true;
        for (int i = 0; i < (int)keep.size() && ok; ++i) {
          if (i == surf_k || keep[i].s == 0 || keep[i].ghost) continue;
          double v = r0 + keep[i].kappa + (t - c[k]) * (t - c[k]);
          if (keep[i].s * v <= 0.0) ok = false;
        }
        if (!ok) continue;
        QP q = bp;
        q.x[k] = t;
        double gn = 0.0;
        for (int i = 0; i < m; ++i) {
          double u = q.x[fr[i]] - c[fr[i]];
          gn += u * u;
        }
        q.w = bp.w * std::sqrt(gn) / std::fabs(t - c[k]);
        out.push_back(q);
        continue;
      }
      roots.clear();
      spts.clear();
      for (const Fn& f : keep) {
        double rho = r0 + f.kappa;
        double t = (rho < 0.0) ? c[k] + sigma * std::sqrt(-rho) : c[k];
        if (f.sing) spts.push_back(t);
        if (!f.ghost && rho < 0.0 && t > a[k] && t < b[k]) roots.push_back({t, f.sing});
      }
      std::sort(roots.begin(), roots.end());
      double t0 = a[k];
      for (size_t j = 0; j <= roots.size(); ++j) {
        double t1 = (j < roots.size()) ? roots[j].first : b[k];
        if (t1 > t0) {
          double mid = 0.5 * (t0 + t1);
          bool ok = true;
          for (const Fn& f : keep) {
            if (f.s == 0 || f.ghost) continue;
            double v = r0 + f.kappa + (mid - c[k]) * (mid - c[k]);
            if (f.s * v <= 0.0) {
              ok = false;
              break;
            }
          }
          if (ok) {
            double SL = -1e300, SR = 1e300;
            for (double sp : spts) {
              if (sp <= t0 && sp > SL) SL = sp;
              if (sp >= t1 && sp < SR) SR = sp;
            }
            pts.clear();
            interval(t0, t1, SL, SR, pts);
            for (auto& pw : pts) {
              QP q = bp;
              q.x[k] = pw.first;
              q.w = bp.w * pw.second;
              out.push_back(q);
            }
          }
        }
        t0 = t1;
      }
    }
  }
};

// ------------------------------------------------------------------------------------------
// problem data
// ------------------------------------------------------------------------------------------
struct Part {
  int cell;
  int sp;        // 0 = A, 1 = B
  double vol;    // |K_{j,s}|
  int cut;       // index into cut data or -1 (full background cell)
  double surf;   // |boundary of K_{j,s}| incl. interface and domain boundary
};

struct CutCell {
  int cell;
  int part[2];
  std::vector<double> G[2], K[2], f[2];  // mass, stiffness, load vector in the cell basis
  std::vector<double> IM, IG;            // interface: int phi_a phi_b, int (grad phi_a . n) phi_b
  double area = 0.0;
};

// a face piece between two parts of the same species, or a boundary piece
struct Face {
  int p, q;    // parts (q = -1 on the domain boundary); p on the lower side (n = +e_d)
  int d;       // direction of the normal
  int sgn;     // boundary: +1/-1 outward normal along e_d
  double meas;
  int mat;     // index into cut face matrices or -1 (uncut: templates)
  int bnd;     // index into boundary load vectors or -1
};

struct Level {
  int nb = 0;
  std::vector<int> part_block;
  std::vector<int32_t> rep;
  std::vector<int8_t> sp, cut;
  std::vector<double> vol;
  std::vector<std::array<double, 6>> box;
  std::vector<int> bp_ptr, bp;        // parts of each block
  std::vector<double> L;              // Cholesky factor of the box-basis mass (Np^2 per block)
  std::vector<int8_t> ident;          // block basis equals the cell Legendre basis
};

struct Problem {
  xp_config cfg;
  int D, N, k, Np, ncell;
  double h;
  std::vector<std::array<int, 3>> modes;
  Rule1 gk1;   // k+1 points: exact for products of degree 2k
  Rule1 gacc;  // k+4 points: non-polynomial data on full cells / faces
  Saye saye;
  Saye saye_hard;  // doubled order for boxes close to the centre in every direction
  std::vector<int> cellpart;  // 2*ncell
  std::vector<int8_t> cellcut;
  std::vector<Part> parts;
  std::vector<CutCell> cuts;
  std::vector<Face> faces;
  std::vector<double> facemats;  // per cut face: 8 Np^2 (Cpp,Cpq,Cqp,Cqq,Ppp,Ppq,Pqp,Pqq)
  std::vector<double> bndvec;    // per boundary face: 2 Np
  std::vector<double> tmpl_face;  // per direction: 8 Np^2
  std::vector<double> tmpl_bnd;   // per (direction, side): 2 Np^2
  std::vector<double> tmpl_stiff; // Np^2
  std::vector<int> agg_target;
  int n_small = 0, n_isolated = 0, n_cut = 0;
  std::vector<Level> levels;
  std::vector<double> ell;  // |dK|/|K| per level-1 block
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<double> val, rhs;
  std::vector<std::vector<int32_t>> agg;
  std::vector<std::vector<double>> Rb;
  double volA = 0, volB = 0, areaI = 0;

  // ---------------- geometry ----------------
  double phi(const double* x) const {
    double s = 0.0;
    for (int d = 0; d < D; ++d) s += (x[d] - cfg.c[d]) * (x[d] - cfg.c[d]);
    return s - cfg.R * cfg.R;
  }
  void cell_ijk(int j, int* ijk) const {
    ijk[0] = j % N;
    ijk[1] = (D > 1) ? (j / N) % N : 0;
    ijk[2] = (D > 2) ? j / (N * N) : 0;
  }
  int cell_index(const int* ijk) const {
    int j = ijk[0];
    if (D > 1) j += N * ijk[1];
    if (D > 2) j += N * N * ijk[2];
    return j;
  }
  void cell_box(int j, double* a, double* b) const {
    int ijk[3];
    cell_ijk(j, ijk);
    for (int d = 0; d < 3; ++d) {
      if (d < D) {
        a[d] = cfg.lo + ijk[d] * h;
        b[d] = a[d] + h;
      } else {
        a[d] = b[d] = 0.0;
      }
    }
  }
  // strict cut test on a box (dims given): min distance < R < max distance
  bool box_cut(const double* a, const double* b, int skip) const {
    double lo = 0, hi = 0;
    for (int d = 0; d < D; ++d) {
      if (d == skip) {
        double u = a[d] - cfg.c[d];
        lo += u * u;
        hi += u * u;
        continue;
      }
      double u = a[d] - cfg.c[d], v = b[d] - cfg.c[d];
      hi += std::max(u * u, v * v);
      lo += (u <= 0 && v >= 0) ? 0.0 : std::min(u * u, v * v);
    }
    double R2 = cfg.R * cfg.R;
    return lo < R2 && R2 < hi;
  }

  // boxes within 1.5 h of the centre in every direction see nearly coincident branch points
  const Saye& saye_for(const double* a, const double* b) const {
    for (int d = 0; d < D; ++d)
      if (std::fabs(0.5 * (a[d] + b[d]) - cfg.c[d]) >= 1.5 * h) return saye;
    return saye_hard;
  }

  // ---------------- basis ----------------
  // orthonormal Legendre basis on box [a,b]: values and (optionally) gradients
  void basis(const double* a, const double* b, const double* x, double* v, double* gr) const {
    double P[3][16], dP[3][16], sc[3][16];
    for (int d = 0; d < D; ++d) {
      double L = b[d] - a[d];
      double t = 2.0 * (x[d] - a[d]) / L - 1.0;
      legendre(k, t, P[d], dP[d]);
      for (int n = 0; n <= k; ++n) sc[d][n] = std::sqrt((2.0 * n + 1.0) / L);
      for (int n = 0; n <= k; ++n) {
        dP[d][n] *= sc[d][n] * 2.0 / L;
        P[d][n] *= sc[d][n];
      }
    }
    for (int m = 0; m < Np; ++m) {
      double val = 1.0;
      for (int d = 0; d < D; ++d) val *= P[d][modes[m][d]];
      v[m] = val;
      if (gr) {
        for (int e = 0; e < D; ++e) {
          double g = 1.0;
          for (int d = 0; d < D; ++d) g *= (d == e) ? dP[d][modes[m][d]] : P[d][modes[m][d]];
          gr[m * 3 + e] = g;
        }
      }
    }
  }

  // T[a][n] = int_cell l^cell_a l^box_n (exact, tensor product of 1-D factors)
  void box_to_cell(const double* box, int cell, double* T) const {
    double ca[3], cb[3];
    cell_box(cell, ca, cb);
    double t1[3][16][16];
    const int q = (int)gk1.u.size();
    double P1[16], dP1[16], P2[16], dP2[16];
    for (int d = 0; d < D; ++d) {
      double bl = box[d], bh = box[3 + d];
      for (int i = 0; i <= k; ++i)
        for (int j = 0; j <= k; ++j) t1[d][i][j] = 0.0;
      for (int g = 0; g < q; ++g) {
        double x = ca[d] + h * gk1.u[g], w = h * gk1.w[g];
        legendre(k, 2.0 * (x - ca[d]) / h - 1.0, P1, dP1);
        legendre(k, 2.0 * (x - bl) / (bh - bl) - 1.0, P2, dP2);
        for (int i = 0; i <= k; ++i)
          for (int j = 0; j <= k; ++j)
            t1[d][i][j] += w * P1[i] * std::sqrt((2.0 * i + 1.0) / h) * P2[j] *
                           std::sqrt((2.0 * j + 1.0) / (bh - bl));
      }
    }
    for (int a2 = 0; a2 < Np; ++a2)
      for (int n = 0; n < Np; ++n) {
        double v = 1.0;
        for (int d = 0; d < D; ++d) v *= t1[d][modes[a2][d]][modes[n][d]];
        T[a2 * Np + n] = v;
      }
  }

  // ---------------- data ----------------
  double gfun(const double* x) const {
    if (cfg.rhs_kind == 0) {
      double g = 1.0;
      for (int d = 0; d < D; ++d) g *= std::cos(M_PI * x[d]);
      return g;
    }
    return 1.0;
  }
  double fsrc(const double* x) const {
    if (cfg.rhs_kind == 2) return 1.0;
    if (cfg.rhs_kind == 1) return -2.0 * D;
    // f = -Laplace(phi g) = -(2D g + 4 (x-c).grad g + phi Laplace g), Laplace g = -D pi^2 g
    double cs[3], sn[3];
    for (int d = 0; d < D; ++d) {
      cs[d] = std::cos(M_PI * x[d]);
      sn[d] = std::sin(M_PI * x[d]);
    }
    double g = 1.0;
    for (int d = 0; d < D; ++d) g *= cs[d];
    double dg = 0.0;
    for (int e = 0; e < D; ++e) {
      double t = -M_PI * sn[e];
      for (int d = 0; d < D; ++d)
        if (d != e) t *= cs[d];
      dg += (x[e] - cfg.c[e]) * t;
    }
    double ph = phi(x);
    return -(2.0 * D * g + 4.0 * dg - D * M_PI * M_PI * ph * g);
  }
  double uexact(const double* x, int sp) const {
    double mu = sp == 0 ? cfg.muA : cfg.muB;
    if (cfg.rhs_kind == 2) return 0.0;
    return phi(x) * gfun(x) / mu;
  }
  double mu(int sp) const { return sp == 0 ? cfg.muA : cfg.muB; }

  void build();
  void cut_cells();
  void build_faces();
  void agglomerate();
  void make_levels();
  void level_bases(Level& L);
  void part_transform(const Level& L, int b, int p, double* C) const;
  void assemble(int level, std::vector<int64_t>& rp, std::vector<int32_t>& cl,
                std::vector<double>& vl, std::vector<double>& rh);
  void transfers();
  double eta_of(int pb, int qb) const;
};

// ------------------------------------------------------------------------------------------
void Problem::cut_cells() {
  cellpart.assign(2 * ncell, -1);
  cellcut.assign(ncell, 0);
  std::vector<int> cutlist;
  for (int j = 0; j < ncell; ++j) {
    double a[3], b[3];
    cell_box(j, a, b);
    if (box_cut(a, b, -1)) {
      cellcut[j] = 1;
      cutlist.push_back(j);
    }
  }
  n_cut = (int)cutlist.size();
  cuts.resize(cutlist.size());
  const int Np2 = Np * Np;
#pragma omp parallel for schedule(dynamic, 4)
  for (int ic = 0; ic < (int)cutlist.size(); ++ic) {
    int j = cutlist[ic];
    CutCell& cc = cuts[ic];
    cc.cell = j;
    double a[3], b[3];
    cell_box(j, a, b);
    int fr[3] = {0, 1, 2};
    double x0[3] = {0, 0, 0};
    std::vector<double> v(Np), gr(Np * 3);
    for (int s = 0; s < 2; ++s) {
      std::vector<QP> rule;
      saye_for(a, b).rec(D, fr, a, b, x0, {{-cfg.R * cfg.R, s == 0 ? -1 : 1, false, false}}, -1, rule);
      cc.G[s].assign(Np2, 0.0);
      cc.K[s].assign(Np2, 0.0);
      cc.f[s].assign(Np, 0.0);
      for (const QP& q : rule) {
        basis(a, b, q.x, v.data(), gr.data());
        double fv = fsrc(q.x) * q.w;
        for (int m = 0; m < Np; ++m) {
          cc.f[s][m] += fv * v[m];
          for (int n = 0; n < Np; ++n) {
            cc.G[s][m * Np + n] += q.w * v[m] * v[n];
            double gg = 0.0;
            for (int d = 0; d < D; ++d) gg += gr[m * 3 + d] * gr[n * 3 + d];
            cc.K[s][m * Np + n] += q.w * gg;
          }
        }
      }
    }
    std::vector<QP> irule;
    saye_for(a, b).rec(D, fr, a, b, x0, {{-cfg.R * cfg.R, 0, false, false}}, 0, irule);
    cc.IM.assign(Np2, 0.0);
    cc.IG.assign(Np2, 0.0);
    for (const QP& q : irule) {
      basis(a, b, q.x, v.data(), gr.data());
      double nrm[3] = {0, 0, 0}, nn = 0.0;
      for (int d = 0; d < D; ++d) {
        nrm[d] = q.x[d] - cfg.c[d];
        nn += nrm[d] * nrm[d];
      }
      nn = std::sqrt(nn);
      for (int d = 0; d < D; ++d) nrm[d] /= nn;
      cc.area += q.w;
      for (int m = 0; m < Np; ++m) {
        double gm = 0.0;
        for (int d = 0; d < D; ++d) gm += gr[m * 3 + d] * nrm[d];
        for (int n = 0; n < Np; ++n) {
          cc.IM[m * Np + n] += q.w * v[m] * v[n];
          cc.IG[m * Np + n] += q.w * gm * v[n];
        }
      }
    }
  }
  // parts
  const double hD = std::pow(h, D);
  const double tiny = 1e-13 * hD;
  std::vector<int> cutidx(ncell, -1);
  for (int ic = 0; ic < (int)cuts.size(); ++ic) cutidx[cuts[ic].cell] = ic;
  parts.clear();
  for (int j = 0; j < ncell; ++j) {
    if (cutidx[j] < 0) {
      double a[3], b[3], xc[3];
      cell_box(j, a, b);
      for (int d = 0; d < 3; ++d) xc[d] = 0.5 * (a[d] + b[d]);
      int sp = phi(xc) < 0.0 ? 0 : 1;
      cellpart[2 * j + sp] = (int)parts.size();
      parts.push_back({j, sp, hD, -1, 0.0});
      (sp == 0 ? volA : volB) += hD;
    } else {
      CutCell& cc = cuts[cutidx[j]];
      cc.part[0] = cc.part[1] = -1;
      for (int s = 0; s < 2; ++s) {
        double vol = 0.0;
        for (int m = 0; m < 1; ++m) vol = cc.G[s][0] * hD;  // mode 0 is 1/sqrt(|K|)
        (s == 0 ? volA : volB) += vol;
        if (vol > tiny) {
          cc.part[s] = (int)parts.size();
          cellpart[2 * j + s] = (int)parts.size();
          parts.push_back({j, s, vol, cutidx[j], 0.0});
        }
      }
      if (cc.part[0] >= 0 && cc.part[1] >= 0) {
        areaI += cc.area;
        parts[cc.part[0]].surf += cc.area;
        parts[cc.part[1]].surf += cc.area;
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
void Problem::build_faces() {
  const int Np2 = Np * Np;
  // templates from a reference pair of full cells
  tmpl_face.assign((size_t)3 * 8 * Np2, 0.0);
  tmpl_bnd.assign((size_t)3 * 2 * 2 * Np2, 0.0);
  tmpl_stiff.assign(Np2, 0.0);
  std::vector<double> v1(Np), g1(3 * Np), v2(Np), g2(3 * Np);
  auto face_integrals = [&](const std::vector<QP>& rule, int d, const double* ap, const double* bp,
                            const double* aq, const double* bq, double* M8) {
    // M8: Cpp, Cpq, Cqp, Cqq, Ppp, Ppq, Pqp, Pqq  [test][trial], normal +e_d from p to q
    std::fill(M8, M8 + 8 * Np2, 0.0);
    for (const QP& q : rule) {
      basis(ap, bp, q.x, v1.data(), g1.data());
      basis(aq, bq, q.x, v2.data(), g2.data());
      double w = q.w;
      for (int t = 0; t < Np; ++t)
        for (int r = 0; r < Np; ++r) {  // t = test, r = trial
          M8[0 * Np2 + t * Np + r] += w * (-0.5 * g1[r * 3 + d] * v1[t] - 0.5 * g1[t * 3 + d] * v1[r]);
          M8[1 * Np2 + t * Np + r] += w * (-0.5 * g2[r * 3 + d] * v1[t] + 0.5 * g1[t * 3 + d] * v2[r]);
          M8[2 * Np2 + t * Np + r] += w * (0.5 * g1[r * 3 + d] * v2[t] - 0.5 * g2[t * 3 + d] * v1[r]);
          M8[3 * Np2 + t * Np + r] += w * (0.5 * g2[r * 3 + d] * v2[t] + 0.5 * g2[t * 3 + d] * v2[r]);
          M8[4 * Np2 + t * Np + r] += w * v1[r] * v1[t];
          M8[5 * Np2 + t * Np + r] += w * (-v2[r] * v1[t]);
          M8[6 * Np2 + t * Np + r] += w * (-v1[r] * v2[t]);
          M8[7 * Np2 + t * Np + r] += w * v2[r] * v2[t];
        }
    }
  };
  auto full_face_rule = [&](int d, double X, const double* a, const double* b, const Rule1& g) {
    std::vector<QP> cur(1);
    for (int e = 0; e < 3; ++e) cur[0].x[e] = 0.0;
    cur[0].x[d] = X;
    cur[0].w = 1.0;
    for (int e = 0; e < D; ++e) {
      if (e == d) continue;
      std::vector<QP> nxt;
      for (const QP& p : cur)
        for (size_t i = 0; i < g.u.size(); ++i) {
          QP r = p;
          r.x[e] = a[e] + (b[e] - a[e]) * g.u[i];
          r.w = p.w * (b[e] - a[e]) * g.w[i];
          nxt.push_back(r);
        }
      cur.swap(nxt);
    }
    return cur;
  };
  {
    double a0[3] = {0, 0, 0}, b0[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) b0[d] = h;
    for (int d = 0; d < D; ++d) {
      double a1[3], b1[3];
      for (int e = 0; e < 3; ++e) {
        a1[e] = a0[e];
        b1[e] = b0[e];
      }
      a1[d] += h;
      b1[d] += h;
      auto rule = full_face_rule(d, h, a0, b0, gk1);
      face_integrals(rule, d, a0, b0, a1, b1, &tmpl_face[(size_t)d * 8 * Np2]);
      for (int side = 0; side < 2; ++side) {
        double X = side == 0 ? 0.0 : h;
        int sg = side == 0 ? -1 : 1;
        auto r2 = full_face_rule(d, X, a0, b0, gk1);
        double* Bc = &tmpl_bnd[((size_t)d * 2 + side) * 2 * Np2];
        double* Bp = Bc + Np2;
        for (const QP& q : r2) {
          basis(a0, b0, q.x, v1.data(), g1.data());
          for (int t = 0; t < Np; ++t)
            for (int r = 0; r < Np; ++r) {
              Bc[t * Np + r] += q.w * (-sg * g1[r * 3 + d] * v1[t] - sg * g1[t * 3 + d] * v1[r]);
              Bp[t * Np + r] += q.w * v1[r] * v1[t];
            }
        }
      }
    }
    // stiffness template
    std::vector<QP> vr(1);
    vr[0].x[0] = vr[0].x[1] = vr[0].x[2] = 0.0;
    vr[0].w = 1.0;
    for (int e = 0; e < D; ++e) {
      std::vector<QP> nxt;
      for (const QP& p : vr)
        for (size_t i = 0; i < gk1.u.size(); ++i) {
          QP r = p;
          r.x[e] = h * gk1.u[i];
          r.w = p.w * h * gk1.w[i];
          nxt.push_back(r);
        }
      vr.swap(nxt);
    }
    for (const QP& q : vr) {
      basis(a0, b0, q.x, v1.data(), g1.data());
      for (int t = 0; t < Np; ++t)
        for (int r = 0; r < Np; ++r) {
          double gg = 0.0;
          for (int d = 0; d < D; ++d) gg += g1[t * 3 + d] * g1[r * 3 + d];
          tmpl_stiff[t * Np + r] += q.w * gg;
        }
    }
  }
  // enumerate faces
  struct FaceJob {
    int j, l, d, side;  // l = -1: boundary, side 0 lower / 1 upper
  };
  std::vector<FaceJob> jobs;
  for (int j = 0; j < ncell; ++j) {
    int ijk[3];
    cell_ijk(j, ijk);
    for (int d = 0; d < D; ++d) {
      if (ijk[d] == 0) jobs.push_back({j, -1, d, 0});
      if (ijk[d] == N - 1) jobs.push_back({j, -1, d, 1});
      else {
        int n2[3] = {ijk[0], ijk[1], ijk[2]};
        n2[d] += 1;
        jobs.push_back({j, cell_index(n2), d, 1});
      }
    }
  }
  // per job, per species: measure and (if cut) matrices
  const double hF = std::pow(h, D - 1);
  struct JobOut {
    double meas[2];
    bool cut;
    std::vector<double> M[2];   // 8 Np^2 (interior) or 2 Np^2 (boundary) matrices if cut
    std::vector<double> bv[2];  // boundary load vectors 2 Np
  };
  std::vector<JobOut> jo(jobs.size());
#pragma omp parallel for schedule(dynamic, 64)
  for (int ij = 0; ij < (int)jobs.size(); ++ij) {
    const FaceJob& fj = jobs[ij];
    JobOut& o = jo[ij];
    double a[3], b[3];
    cell_box(fj.j, a, b);
    double X = fj.side == 0 ? a[fj.d] : b[fj.d];
    double fa[3], fb[3];
    for (int e = 0; e < 3; ++e) {
      fa[e] = a[e];
      fb[e] = b[e];
    }
    fa[fj.d] = fb[fj.d] = X;
    o.cut = box_cut(fa, fb, fj.d);
    o.meas[0] = o.meas[1] = 0.0;
    std::vector<QP> rules[2];
    if (o.cut) {
      int fr[3], m = 0;
      for (int e = 0; e < D; ++e)
        if (e != fj.d) fr[m++] = e;
      double x0[3] = {0, 0, 0};
      x0[fj.d] = X;
      double kap = -cfg.R * cfg.R + (X - cfg.c[fj.d]) * (X - cfg.c[fj.d]);
      for (int s = 0; s < 2; ++s) {
        saye_for(a, b).rec(m, fr, fa, fb, x0, {{kap, s == 0 ? -1 : 1, false, false}}, -1, rules[s]);
        for (const QP& q : rules[s]) o.meas[s] += q.w;
      }
    } else {
      double xc[3];
      for (int e = 0; e < 3; ++e) xc[e] = 0.5 * (fa[e] + fb[e]);
      int sp = phi(xc) < 0.0 ? 0 : 1;
      o.meas[sp] = hF;
    }
    std::vector<double> vv(Np), gg(3 * Np);
    for (int s = 0; s < 2; ++s) {
      if (!(o.meas[s] > 1e-13 * hF)) continue;
      if (fj.l >= 0) {
        if (o.cut) {
          double la[3], lb[3];
          cell_box(fj.l, la, lb);
          o.M[s].resize(8 * Np2);
          // local copies of scratch for thread safety
          std::vector<double> s1(Np), s2(3 * Np), s3(Np), s4(3 * Np);
          std::fill(o.M[s].begin(), o.M[s].end(), 0.0);
          for (const QP& q : rules[s]) {
            basis(a, b, q.x, s1.data(), s2.data());
            basis(la, lb, q.x, s3.data(), s4.data());
            double w = q.w;
            int d = fj.d;
            for (int t = 0; t < Np; ++t)
              for (int r = 0; r < Np; ++r) {
                o.M[s][0 * Np2 + t * Np + r] += w * (-0.5 * s2[r * 3 + d] * s1[t] - 0.5 * s2[t * 3 + d] * s1[r]);
                o.M[s][1 * Np2 + t * Np + r] += w * (-0.5 * s4[r * 3 + d] * s1[t] + 0.5 * s2[t * 3 + d] * s3[r]);
                o.M[s][2 * Np2 + t * Np + r] += w * (0.5 * s2[r * 3 + d] * s3[t] - 0.5 * s4[t * 3 + d] * s1[r]);
                o.M[s][3 * Np2 + t * Np + r] += w * (0.5 * s4[r * 3 + d] * s3[t] + 0.5 * s4[t * 3 + d] * s3[r]);
                o.M[s][4 * Np2 + t * Np + r] += w * s1[r] * s1[t];
                o.M[s][5 * Np2 + t * Np + r] += w * (-s3[r] * s1[t]);
                o.M[s][6 * Np2 + t * Np + r] += w * (-s1[r] * s3[t]);
                o.M[s][7 * Np2 + t * Np + r] += w * s3[r] * s3[t];
              }
          }
        }
      } else {
        int sg = fj.side == 0 ? -1 : 1;
        std::vector<QP> r2;
        if (o.cut) r2 = rules[s];
        else r2 = full_face_rule(fj.d, X, fa, fb, gacc);
        if (o.cut) {
          o.M[s].assign(2 * Np2, 0.0);
        }
        o.bv[s].assign(2 * Np, 0.0);
        for (const QP& q : r2) {
          basis(a, b, q.x, vv.data(), gg.data());
          double gd = uexact(q.x, s);
          for (int t = 0; t < Np; ++t) {
            o.bv[s][t] += q.w * gd * (-sg * gg[t * 3 + fj.d]);
            o.bv[s][Np + t] += q.w * gd * vv[t];
            if (o.cut)
              for (int r = 0; r < Np; ++r) {
                o.M[s][t * Np + r] += q.w * (-sg * gg[r * 3 + fj.d] * vv[t] - sg * gg[t * 3 + fj.d] * vv[r]);
                o.M[s][Np2 + t * Np + r] += q.w * vv[r] * vv[t];
              }
          }
        }
      }
    }
  }
  (void)face_integrals;
  // collect face pieces between existing parts
  faces.clear();
  facemats.clear();
  bndvec.clear();
  for (size_t ij = 0; ij < jobs.size(); ++ij) {
    const FaceJob& fj = jobs[ij];
    JobOut& o = jo[ij];
    for (int s = 0; s < 2; ++s) {
      if (!(o.meas[s] > 1e-13 * hF)) continue;
      int p = cellpart[2 * fj.j + s];
      if (p < 0) continue;
      Face f;
      f.d = fj.d;
      f.meas = o.meas[s];
      f.mat = -1;
      f.bnd = -1;
      if (fj.l >= 0) {
        int q = cellpart[2 * fj.l + s];
        if (q < 0) continue;
        f.p = p;
        f.q = q;
        f.sgn = 1;
        if (o.cut) {
          f.mat = (int)(facemats.size() / (8 * Np2));
          facemats.insert(facemats.end(), o.M[s].begin(), o.M[s].end());
        }
        parts[p].surf += f.meas;
        parts[q].surf += f.meas;
      } else {
        f.p = p;
        f.q = -1;
        f.sgn = fj.side == 0 ? -1 : 1;
        f.bnd = (int)(bndvec.size() / (2 * Np));
        bndvec.insert(bndvec.end(), o.bv[s].begin(), o.bv[s].end());
        if (o.cut) {
          f.mat = (int)(facemats.size() / (8 * Np2));
          std::vector<double> pad(8 * Np2, 0.0);
          std::copy(o.M[s].begin(), o.M[s].end(), pad.begin());
          facemats.insert(facemats.end(), pad.begin(), pad.end());
        }
        parts[p].surf += f.meas;
      }
      faces.push_back(f);
    }
  }
}

// ------------------------------------------------------------------------------------------
// agglomeration map A_alpha (sec. 2.3): every part with 0 < fraction <= alpha is attached to
// its largest same-species neighbour (a neighbour shares a face piece of positive measure).
// Among neighbours, parts that are not small themselves are preferred; ties go to the smaller
// background cell index.
void Problem::agglomerate() {
  const double hD = std::pow(h, D);
  std::vector<std::vector<int>> nbr(parts.size());
  for (const Face& f : faces)
    if (f.q >= 0) {
      nbr[f.p].push_back(f.q);
      nbr[f.q].push_back(f.p);
    }
  agg_target.assign(parts.size(), -1);
  n_small = n_isolated = 0;
  for (int p = 0; p < (int)parts.size(); ++p) {
    double frac = parts[p].vol / hD;
    if (!(frac <= cfg.alpha)) continue;
    ++n_small;
    int best = -1;
    bool best_big = false;
    for (int q : nbr[p]) {
      bool big = parts[q].vol / hD > cfg.alpha;
      if (best < 0 || (big && !best_big) ||
          (big == best_big && (parts[q].vol > parts[best].vol ||
                               (parts[q].vol == parts[best].vol && parts[q].cell < parts[best].cell)))) {
        best = q;
        best_big = big;
      }
    }
    if (best < 0) ++n_isolated;
    agg_target[p] = best;
  }
}

struct DSU {
  std::vector<int> p;
  explicit DSU(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int find(int x) {
    while (p[x] != x) {
      p[x] = p[p[x]];
      x = p[x];
    }
    return x;
  }
  void unite(int a, int b) {
    a = find(a);
    b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

// ------------------------------------------------------------------------------------------
// level lambda: connected components of (A^lambda)^X U A_alpha (sec. 3.1). The background
// aggregation groups 2 cells per direction per level; an odd trailing cell joins the last
// group of its row.
void Problem::make_levels() {
  levels.clear();
  const int np = (int)parts.size();
  std::vector<int> grp(ncell);  // group index per direction, packed
  std::vector<int> gcoord(3 * ncell);
  for (int j = 0; j < ncell; ++j) {
    int ijk[3];
    cell_ijk(j, ijk);
    for (int d = 0; d < 3; ++d) gcoord[3 * j + d] = ijk[d];
  }
  int ng[3] = {N, D > 1 ? N : 1, D > 2 ? N : 1};
  int prev_nb = -1;
  for (int lev = 1; lev <= cfg.max_levels; ++lev) {
    if (lev > 1) {
      bool any = false;
      int ng2[3];
      for (int d = 0; d < 3; ++d) {
        ng2[d] = ng[d] >= 2 ? ng[d] / 2 : 1;
        if (ng2[d] != ng[d]) any = true;
      }
      if (!any) break;
      for (int j = 0; j < ncell; ++j)
        for (int d = 0; d < 3; ++d) gcoord[3 * j + d] = std::min(gcoord[3 * j + d] / 2, ng2[d] - 1);
      for (int d = 0; d < 3; ++d) ng[d] = ng2[d];
    }
    DSU dsu(np);
    for (int p = 0; p < np; ++p)
      if (agg_target[p] >= 0) dsu.unite(p, agg_target[p]);
    if (lev > 1) {
      for (int j = 0; j < ncell; ++j) {
        int ijk[3];
        cell_ijk(j, ijk);
        for (int d = 0; d < D; ++d) {
          if (ijk[d] + 1 >= N) continue;
          int n2[3] = {ijk[0], ijk[1], ijk[2]};
          n2[d] += 1;
          int l = cell_index(n2);
          bool same = true;
          for (int e = 0; e < 3; ++e)
            if (gcoord[3 * j + e] != gcoord[3 * l + e]) same = false;
          if (!same) continue;
          for (int s = 0; s < 2; ++s) {
            int p = cellpart[2 * j + s], q = cellpart[2 * l + s];
            if (p >= 0 && q >= 0) dsu.unite(p, q);
          }
        }
      }
    }
    // blocks: order by (minimum background cell index, species)
    std::vector<int> root(np), rep(np, INT32_MAX);
    for (int p = 0; p < np; ++p) {
      root[p] = dsu.find(p);
      rep[root[p]] = std::min(rep[root[p]], parts[p].cell);
    }
    std::vector<std::pair<long long, int>> keys;
    for (int p = 0; p < np; ++p)
      if (root[p] == p) keys.push_back({(long long)rep[p] * 2 + parts[p].sp, p});
    std::sort(keys.begin(), keys.end());
    Level L;
    L.nb = (int)keys.size();
    std::vector<int> rootblk(np, -1);
    for (int i = 0; i < L.nb; ++i) rootblk[keys[i].second] = i;
    L.part_block.resize(np);
    for (int p = 0; p < np; ++p) L.part_block[p] = rootblk[root[p]];
    L.rep.resize(L.nb);
    L.sp.resize(L.nb);
    L.cut.assign(L.nb, 0);
    L.vol.assign(L.nb, 0.0);
    for (int i = 0; i < L.nb; ++i) {
      L.rep[i] = (int32_t)(keys[i].first / 2);
      L.sp[i] = (int8_t)(keys[i].first % 2);
    }
    L.bp_ptr.assign(L.nb + 1, 0);
    for (int p = 0; p < np; ++p) L.bp_ptr[L.part_block[p] + 1]++;
    for (int i = 0; i < L.nb; ++i) L.bp_ptr[i + 1] += L.bp_ptr[i];
    L.bp.resize(np);
    {
      std::vector<int> pos(L.bp_ptr.begin(), L.bp_ptr.end() - 1);
      for (int p = 0; p < np; ++p) L.bp[pos[L.part_block[p]]++] = p;
    }
    for (int p = 0; p < np; ++p) {
      int bl = L.part_block[p];
      L.vol[bl] += parts[p].vol;
      if (parts[p].cut >= 0) L.cut[bl] = 1;
    }
    level_bases(L);
    const int nb = L.nb;
    levels.push_back(std::move(L));
    if ((long long)nb * Np <= cfg.max_coarse_dof) break;
    if (nb == prev_nb) {
      levels.pop_back();
      break;
    }
    prev_nb = nb;
  }
}

// bounding box and the Cholesky factor of the mass matrix of the box Legendre basis
// restricted to the species domain of the block (re-orthonormalisation S, Eq. XdgMgBasis)
void Problem::level_bases(Level& L) {
  const int Np2 = Np * Np;
  L.box.resize(L.nb);
  L.L.assign((size_t)L.nb * Np2, 0.0);
  L.ident.assign(L.nb, 0);
  std::vector<int> fail(L.nb, 0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int bl = 0; bl < L.nb; ++bl) {
    std::array<double, 6> bx;
    for (int d = 0; d < 3; ++d) {
      bx[d] = 1e300;
      bx[3 + d] = -1e300;
    }
    for (int i = L.bp_ptr[bl]; i < L.bp_ptr[bl + 1]; ++i) {
      double a[3], b[3];
      cell_box(parts[L.bp[i]].cell, a, b);
      for (int d = 0; d < 3; ++d) {
        bx[d] = std::min(bx[d], a[d]);
        bx[3 + d] = std::max(bx[3 + d], b[d]);
      }
    }
    L.box[bl] = bx;
    double* Lm = &L.L[(size_t)bl * Np2];
    int np_in = L.bp_ptr[bl + 1] - L.bp_ptr[bl];
    if (np_in == 1 && parts[L.bp[L.bp_ptr[bl]]].cut < 0) {
      for (int i = 0; i < Np; ++i) Lm[i * Np + i] = 1.0;
      L.ident[bl] = 1;
      continue;
    }
    std::vector<double> T(Np2), GT(Np2), Ms(Np2, 0.0);
    for (int i = L.bp_ptr[bl]; i < L.bp_ptr[bl + 1]; ++i) {
      const Part& P = parts[L.bp[i]];
      box_to_cell(bx.data(), P.cell, T.data());
      if (P.cut < 0) {
        gemm_tn(Np, Np, Np, T.data(), T.data(), Ms.data(), true);
      } else {
        gemm_nn(Np, Np, Np, cuts[P.cut].G[P.sp].data(), T.data(), GT.data());
        gemm_tn(Np, Np, Np, T.data(), GT.data(), Ms.data(), true);
      }
    }
    // symmetrise
    for (int i = 0; i < Np; ++i)
      for (int j = 0; j < i; ++j) {
        double s = 0.5 * (Ms[i * Np + j] + Ms[j * Np + i]);
        Ms[i * Np + j] = Ms[j * Np + i] = s;
      }
    if (!cholesky(Np, Ms.data())) fail[bl] = 1;
    std::copy(Ms.begin(), Ms.end(), Lm);
  }
  for (int bl = 0; bl < L.nb; ++bl)
    if (fail[bl]) throw std::runtime_error("block mass matrix not positive definite (block " +
                                           std::to_string(bl) + ")");
}

// C = T(box_b -> cell of p) L_b^{-T}: coefficients of the level basis of block b in the cell
// Legendre basis of part p
void Problem::part_transform(const Level& L, int b, int p, double* C) const {
  const int Np2 = Np * Np;
  std::vector<double> T(Np2);
  box_to_cell(L.box[b].data(), parts[p].cell, T.data());
  right_solve_LT(Np, Np, &L.L[(size_t)b * Np2], T.data(), C);
}

double Problem::eta_of(int pb, int qb) const {
  double e = ell[pb];
  if (qb >= 0) e = std::max(e, ell[qb]);
  return cfg.ceta * (k + 1.0) * (k + D) / D * e;
}

// ------------------------------------------------------------------------------------------
// assembly of a_sip and b in the basis of a level: M = sum over contributions C_p^T X C_q
void Problem::assemble(int level, std::vector<int64_t>& rp, std::vector<int32_t>& cl,
                       std::vector<double>& vl, std::vector<double>& rh) {
  const Level& L = levels[level - 1];
  const Level& L1 = levels[0];
  const int Np2 = Np * Np;
  const int np = (int)parts.size();
  // per-part transforms (identity flagged)
  std::vector<int> cidx(np, -1);
  std::vector<double> Cs;
  {
    std::vector<int> need;
    for (int p = 0; p < np; ++p) {
      int bl = L.part_block[p];
      if (!L.ident[bl]) {
        cidx[p] = (int)need.size();
        need.push_back(p);
      }
    }
    Cs.resize((size_t)need.size() * Np2);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < (int)need.size(); ++i)
      part_transform(L, L.part_block[need[i]], need[i], &Cs[(size_t)i * Np2]);
  }
  // sparsity: pairs of blocks
  std::vector<std::vector<int>> rows(L.nb);
  auto pair = [&](int p, int q) {
    rows[L.part_block[p]].push_back(L.part_block[q]);
  };
  for (int p = 0; p < np; ++p) pair(p, p);
  for (const CutCell& cc : cuts)
    if (cc.part[0] >= 0 && cc.part[1] >= 0) {
      pair(cc.part[0], cc.part[1]);
      pair(cc.part[1], cc.part[0]);
    }
  for (const Face& f : faces)
    if (f.q >= 0) {
      pair(f.p, f.q);
      pair(f.q, f.p);
    }
  rp.assign(L.nb + 1, 0);
  for (int i = 0; i < L.nb; ++i) {
    std::sort(rows[i].begin(), rows[i].end());
    rows[i].erase(std::unique(rows[i].begin(), rows[i].end()), rows[i].end());
    rp[i + 1] = rp[i] + (int64_t)rows[i].size();
  }
  cl.resize(rp[L.nb]);
  for (int i = 0; i < L.nb; ++i)
    std::copy(rows[i].begin(), rows[i].end(), cl.begin() + rp[i]);
  rows.clear();
  rows.shrink_to_fit();
  vl.assign((size_t)rp[L.nb] * Np2, 0.0);
  rh.assign((size_t)L.nb * Np, 0.0);
  auto find = [&](int bi, int bj) -> double* {
    auto b = cl.begin() + rp[bi], e = cl.begin() + rp[bi + 1];
    auto it = std::lower_bound(b, e, bj);
    return &vl[(size_t)(it - cl.begin()) * Np2];
  };
  std::vector<double> tmp(Np2), tmp2(Np2);
  // add C_p^T X C_q (X[test][trial]) into block (B(p), B(q)) scaled by s
  auto add = [&](int p, int q, const double* X, double s) {
    double* dst = find(L.part_block[p], L.part_block[q]);
    const double* Cp = cidx[p] >= 0 ? &Cs[(size_t)cidx[p] * Np2] : nullptr;
    const double* Cq = cidx[q] >= 0 ? &Cs[(size_t)cidx[q] * Np2] : nullptr;
    const double* Y = X;
    if (Cq) {
      gemm_nn(Np, Np, Np, X, Cq, tmp.data());
      Y = tmp.data();
    }
    if (Cp) {
      gemm_tn(Np, Np, Np, Cp, Y, tmp2.data(), false);
      Y = tmp2.data();
    }
    for (int i = 0; i < Np2; ++i) dst[i] += s * Y[i];
  };
  auto addv = [&](int p, const double* v, double s) {
    double* dst = &rh[(size_t)L.part_block[p] * Np];
    const double* Cp = cidx[p] >= 0 ? &Cs[(size_t)cidx[p] * Np2] : nullptr;
    for (int n = 0; n < Np; ++n) {
      double t = 0.0;
      if (Cp)
        for (int a = 0; a < Np; ++a) t += Cp[a * Np + n] * v[a];
      else
        t = v[n];
      dst[n] += s * t;
    }
  };
  const double hD = std::pow(h, D);
  std::vector<double> fv(Np), vv(Np);
  // volume terms and volume load
  for (int p = 0; p < np; ++p) {
    const Part& P = parts[p];
    double m = mu(P.sp);
    if (P.cut < 0) {
      add(p, p, tmpl_stiff.data(), m);
      // load vector with a k+4 point rule
      double a[3], b[3];
      cell_box(P.cell, a, b);
      std::fill(fv.begin(), fv.end(), 0.0);
      const int q = (int)gacc.u.size();
      int idx[3] = {0, 0, 0};
      int tot = 1;
      for (int d = 0; d < D; ++d) tot *= q;
      for (int t = 0; t < tot; ++t) {
        int r = t;
        double x[3] = {0, 0, 0}, w = 1.0;
        for (int d = 0; d < D; ++d) {
          idx[d] = r % q;
          r /= q;
          x[d] = a[d] + h * gacc.u[idx[d]];
          w *= h * gacc.w[idx[d]];
        }
        basis(a, b, x, vv.data(), nullptr);
        double f = fsrc(x) * w;
        for (int n = 0; n < Np; ++n) fv[n] += f * vv[n];
      }
      addv(p, fv.data(), 1.0);
    } else {
      const CutCell& cc = cuts[P.cut];
      add(p, p, cc.K[P.sp].data(), m);
      addv(p, cc.f[P.sp].data(), 1.0);
    }
  }
  (void)hD;
  // interface terms (normal from A to B)
  std::vector<double> X(Np2);
  for (const CutCell& cc : cuts) {
    int pa = cc.part[0], pb = cc.part[1];
    if (pa < 0 || pb < 0) continue;
    double mA = cfg.muA, mB = cfg.muB, mmax = std::max(mA, mB);
    double eta = eta_of(L1.part_block[pa], L1.part_block[pb]);
    const double* IM = cc.IM.data();
    const double* IG = cc.IG.data();
    for (int t = 0; t < Np; ++t)
      for (int r = 0; r < Np; ++r)
        X[t * Np + r] = -0.5 * mA * (IG[r * Np + t] + IG[t * Np + r]) + eta * mmax * IM[t * Np + r];
    add(pa, pa, X.data(), 1.0);
    for (int t = 0; t < Np; ++t)
      for (int r = 0; r < Np; ++r)
        X[t * Np + r] = -0.5 * mB * IG[r * Np + t] + 0.5 * mA * IG[t * Np + r] - eta * mmax * IM[t * Np + r];
    add(pa, pb, X.data(), 1.0);
    for (int t = 0; t < Np; ++t)
      for (int r = 0; r < Np; ++r)
        X[t * Np + r] = -0.5 * mB * IG[t * Np + r] + 0.5 * mA * IG[r * Np + t] - eta * mmax * IM[r * Np + t];
    add(pb, pa, X.data(), 1.0);
    for (int t = 0; t < Np; ++t)
      for (int r = 0; r < Np; ++r)
        X[t * Np + r] = 0.5 * mB * (IG[r * Np + t] + IG[t * Np + r]) + eta * mmax * IM[t * Np + r];
    add(pb, pb, X.data(), 1.0);
  }
  // faces
  for (const Face& f : faces) {
    double m = mu(parts[f.p].sp);
    if (f.q >= 0) {
      double eta = eta_of(L1.part_block[f.p], L1.part_block[f.q]);
      const double* M8 = f.mat >= 0 ? &facemats[(size_t)f.mat * 8 * Np2]
                                    : &tmpl_face[(size_t)f.d * 8 * Np2];
      const int pr[4][2] = {{f.p, f.p}, {f.p, f.q}, {f.q, f.p}, {f.q, f.q}};
      for (int c = 0; c < 4; ++c) {
        for (int i = 0; i < Np2; ++i) X[i] = m * (M8[c * Np2 + i] + eta * M8[(4 + c) * Np2 + i]);
        add(pr[c][0], pr[c][1], X.data(), 1.0);
      }
    } else {
      double eta = eta_of(L1.part_block[f.p], -1);
      const double* B2 = f.mat >= 0 ? &facemats[(size_t)f.mat * 8 * Np2]
                                    : &tmpl_bnd[((size_t)f.d * 2 + (f.sgn > 0 ? 1 : 0)) * 2 * Np2];
      for (int i = 0; i < Np2; ++i) X[i] = m * (B2[i] + eta * B2[Np2 + i]);
      add(f.p, f.p, X.data(), 1.0);
      const double* bv = &bndvec[(size_t)f.bnd * 2 * Np];
      for (int n = 0; n < Np; ++n) fv[n] = m * (bv[n] + eta * bv[Np + n]);
      addv(f.p, fv.data(), 1.0);
    }
  }
  // a_sip is symmetric; the transforms C_p^T X C_q of ill-conditioned cut-cell bases leave
  // rounding-level asymmetry, removed by averaging M_ij with M_ji^T
  for (int i = 0; i < L.nb; ++i)
    for (int64_t z = rp[i]; z < rp[i + 1]; ++z) {
      int j = cl[z];
      if (j < i) continue;
      double* Mij = &vl[(size_t)z * Np2];
      double* Mji = find(j, i);
      for (int a = 0; a < Np; ++a)
        for (int c2 = 0; c2 < Np; ++c2) {
          if (j == i && c2 <= a) continue;
          double v = 0.5 * (Mij[a * Np + c2] + Mji[c2 * Np + a]);
          Mij[a * Np + c2] = v;
          Mji[c2 * Np + a] = v;
        }
    }
}

// ------------------------------------------------------------------------------------------
// R_f = L_f^{-1} [ sum_{p in f} T(box_f -> p)^T G_p T(box_C -> p) ] L_C^{-T}   (Eq. XDGrestrictionMatrix)
void Problem::transfers() {
  agg.clear();
  Rb.clear();
  const int Np2 = Np * Np;
  for (size_t lv = 0; lv + 1 < levels.size(); ++lv) {
    const Level& F = levels[lv];
    const Level& C = levels[lv + 1];
    std::vector<int32_t> ag(F.nb);
    std::vector<double> R((size_t)F.nb * Np2);
#pragma omp parallel for schedule(dynamic, 256)
    for (int f = 0; f < F.nb; ++f) {
      int p0 = F.bp[F.bp_ptr[f]];
      int cb = C.part_block[p0];
      ag[f] = cb;
      std::vector<double> Tf(Np2), Tc(Np2), GT(Np2), S(Np2, 0.0), X(Np2);
      for (int i = F.bp_ptr[f]; i < F.bp_ptr[f + 1]; ++i) {
        const Part& P = parts[F.bp[i]];
        box_to_cell(F.box[f].data(), P.cell, Tf.data());
        box_to_cell(C.box[cb].data(), P.cell, Tc.data());
        if (P.cut < 0) {
          gemm_tn(Np, Np, Np, Tf.data(), Tc.data(), S.data(), true);
        } else {
          gemm_nn(Np, Np, Np, cuts[P.cut].G[P.sp].data(), Tc.data(), GT.data());
          gemm_tn(Np, Np, Np, Tf.data(), GT.data(), S.data(), true);
        }
      }
      left_solve_L(Np, Np, &F.L[(size_t)f * Np2], S.data());
      right_solve_LT(Np, Np, &C.L[(size_t)cb * Np2], S.data(), X.data());
      std::copy(X.begin(), X.end(), R.begin() + (size_t)f * Np2);
    }
    agg.push_back(std::move(ag));
    Rb.push_back(std::move(R));
  }
}

void Problem::build() {
  D = cfg.D;
  N = cfg.N;
  k = cfg.k;
  if (D < 2 || D > 3) throw std::runtime_error("D must be 2 or 3");
  if (k < 0 || k > 6) throw std::runtime_error("k must be in 0..6");
  if (N < 1) throw std::runtime_error("N must be >= 1");
  if (cfg.max_levels < 1) cfg.max_levels = 1;
  h = (cfg.hi - cfg.lo) / N;
  ncell = 1;
  for (int d = 0; d < D; ++d) ncell *= N;
  modes.clear();
  for (int p = 0; p <= k; ++p) {
    if (D == 2) {
      for (int j = 0; j <= p; ++j) modes.push_back({p - j, j, 0});
    } else {
      for (int j2 = 0; j2 <= p; ++j2)
        for (int j1 = 0; j1 <= p - j2; ++j1) modes.push_back({p - j1 - j2, j1, j2});
    }
  }
  Np = (int)modes.size();
  gk1 = gauss01(k + 1);
  gacc = gauss01(k + 4);
  int q = cfg.quad_q > 0 ? cfg.quad_q : std::max(2 * k + 4, 10);
  saye.D = D;
  for (int d = 0; d < 3; ++d) saye.c[d] = d < D ? cfg.c[d] : 0.0;
  saye.g = gauss01(q);
  saye_hard = saye;
  saye_hard.g = gauss01(std::max(2 * q, 24));
  cut_cells();
  build_faces();
  agglomerate();
  make_levels();
  // |dK|/|K| of level-1 blocks: faces between parts of the same block are interior
  const Level& L1 = levels[0];
  std::vector<double> surf(L1.nb, 0.0), vol(L1.nb, 0.0);
  for (int p = 0; p < (int)parts.size(); ++p) {
    surf[L1.part_block[p]] += parts[p].surf;
    vol[L1.part_block[p]] += parts[p].vol;
  }
  for (const Face& f : faces)
    if (f.q >= 0 && L1.part_block[f.p] == L1.part_block[f.q]) surf[L1.part_block[f.p]] -= 2.0 * f.meas;
  ell.resize(L1.nb);
  for (int b = 0; b < L1.nb; ++b) ell[b] = surf[b] / vol[b];
  int64_t dummy = 0;
  (void)dummy;
  assemble(1, row_ptr, col, val, rhs);
  transfers();
}

}  // namespace

// ------------------------------------------------------------------------------------------
extern "C" {

void* xp_build(const xp_config* cfg, char* err, int errlen) {
  Problem* P = new Problem();
  P->cfg = *cfg;
#ifdef _OPENMP
  if (cfg->nthreads > 0) omp_set_num_threads(cfg->nthreads);
#endif
  try {
    P->build();
  } catch (const std::exception& e) {
    if (err && errlen > 0) std::snprintf(err, errlen, "%s", e.what());
    delete P;
    return nullptr;
  }
  return P;
}

void xp_free(void* h) { delete static_cast<Problem*>(h); }

void xp_get_info(void* h, xp_info* o) {
  Problem* P = static_cast<Problem*>(h);
  o->D = P->D;
  o->N = P->N;
  o->k = P->k;
  o->Np = P->Np;
  o->n_levels = (int)P->levels.size();
  o->n_cells = P->ncell;
  o->n_cut_cells = P->n_cut;
  o->n_parts = (int)P->parts.size();
  o->n_small = P->n_small;
  o->n_isolated = P->n_isolated;
  o->nnzb1 = P->row_ptr.empty() ? 0 : P->row_ptr.back();
  o->volA = P->volA;
  o->volB = P->volB;
  o->areaI = P->areaI;
  o->h = P->h;
}

static const Level* lev(void* h, int level) {
  Problem* P = static_cast<Problem*>(h);
  if (level < 1 || level > (int)P->levels.size()) return nullptr;
  return &P->levels[level - 1];
}
int xp_level_nb(void* h, int level) {
  const Level* L = lev(h, level);
  return L ? L->nb : -1;
}
const int32_t* xp_level_rep(void* h, int level) {
  const Level* L = lev(h, level);
  return L ? L->rep.data() : nullptr;
}
const int8_t* xp_level_species(void* h, int level) {
  const Level* L = lev(h, level);
  return L ? L->sp.data() : nullptr;
}
const double* xp_level_volume(void* h, int level) {
  const Level* L = lev(h, level);
  return L ? L->vol.data() : nullptr;
}
const int8_t* xp_level_cut(void* h, int level) {
  const Level* L = lev(h, level);
  return L ? L->cut.data() : nullptr;
}
const int64_t* xp_row_ptr(void* h) { return static_cast<Problem*>(h)->row_ptr.data(); }
const int32_t* xp_col(void* h) { return static_cast<Problem*>(h)->col.data(); }
const double* xp_val(void* h) { return static_cast<Problem*>(h)->val.data(); }
const double* xp_rhs(void* h) { return static_cast<Problem*>(h)->rhs.data(); }
const int32_t* xp_agg(void* h, int level) {
  Problem* P = static_cast<Problem*>(h);
  if (level < 1 || level >= (int)P->levels.size()) return nullptr;
  return P->agg[level - 1].data();
}
const double* xp_R(void* h, int level) {
  Problem* P = static_cast<Problem*>(h);
  if (level < 1 || level >= (int)P->levels.size()) return nullptr;
  return P->Rb[level - 1].data();
}

int xp_assemble_level(void* h, int level, int64_t** row_ptr, int32_t** col, double** val,
                      double** rhs, int64_t* nnzb) {
  Problem* P = static_cast<Problem*>(h);
  if (level < 1 || level > (int)P->levels.size()) return -1;
  std::vector<int64_t> rp;
  std::vector<int32_t> cl;
  std::vector<double> vl, rh;
  P->assemble(level, rp, cl, vl, rh);
  *row_ptr = (int64_t*)std::malloc(rp.size() * sizeof(int64_t));
  *col = (int32_t*)std::malloc(std::max<size_t>(cl.size(), 1) * sizeof(int32_t));
  *val = (double*)std::malloc(std::max<size_t>(vl.size(), 1) * sizeof(double));
  *rhs = (double*)std::malloc(std::max<size_t>(rh.size(), 1) * sizeof(double));
  std::copy(rp.begin(), rp.end(), *row_ptr);
  std::copy(cl.begin(), cl.end(), *col);
  std::copy(vl.begin(), vl.end(), *val);
  std::copy(rh.begin(), rh.end(), *rhs);
  *nnzb = rp.back();
  return 0;
}
void xp_release(void* p) { std::free(p); }

int xp_l2_error(void* h, const double* x, double* err2, double* norm2) {
  Problem* P = static_cast<Problem*>(h);
  if (P->cfg.rhs_kind == 2) return -1;
  const Level& L = P->levels[0];
  const int Np = P->Np, Np2 = Np * Np, D = P->D;
  // y_B = L_B^{-T} x_B: coefficients of u_h in the box Legendre basis of block B
  std::vector<double> y((size_t)L.nb * Np);
  for (int b = 0; b < L.nb; ++b) {
    const double* Lm = &L.L[(size_t)b * Np2];
    const double* xb = x + (size_t)b * Np;
    double* yb = &y[(size_t)b * Np];
    for (int i = Np - 1; i >= 0; --i) {
      double s = xb[i];
      for (int p = i + 1; p < Np; ++p) s -= Lm[p * Np + i] * yb[p];
      yb[i] = s / Lm[i * Np + i];
    }
  }
  double e2 = 0.0, n2 = 0.0;
  const int np = (int)P->parts.size();
#pragma omp parallel for reduction(+ : e2, n2) schedule(dynamic, 64)
  for (int p = 0; p < np; ++p) {
    const Part& Pt = P->parts[p];
    int b = L.part_block[p];
    double a[3], bb[3];
    P->cell_box(Pt.cell, a, bb);
    std::vector<QP> rule;
    if (Pt.cut >= 0) {
      int fr[3] = {0, 1, 2};
      double x0[3] = {0, 0, 0};
      P->saye_for(a, bb).rec(D, fr, a, bb, x0, {{-P->cfg.R * P->cfg.R, Pt.sp == 0 ? -1 : 1, false, false}}, -1, rule);
    } else {
      const Rule1& g = P->gacc;
      rule.resize(1);
      rule[0].x[0] = rule[0].x[1] = rule[0].x[2] = 0.0;
      rule[0].w = 1.0;
      for (int d = 0; d < D; ++d) {
        std::vector<QP> nxt;
        for (const QP& q : rule)
          for (size_t i = 0; i < g.u.size(); ++i) {
            QP r = q;
            r.x[d] = a[d] + P->h * g.u[i];
            r.w = q.w * P->h * g.w[i];
            nxt.push_back(r);
          }
        rule.swap(nxt);
      }
    }
    std::vector<double> v(Np);
    const double* bx = L.box[b].data();
    for (const QP& q : rule) {
      P->basis(bx, bx + 3, q.x, v.data(), nullptr);
      double uh = 0.0;
      for (int n = 0; n < Np; ++n) uh += y[(size_t)b * Np + n] * v[n];
      double ue = P->uexact(q.x, Pt.sp);
      e2 += q.w * (uh - ue) * (uh - ue);
      n2 += q.w * ue * ue;
    }
  }
  *err2 = e2;
  *norm2 = n2;
  return 0;
}

static void cell_features(const Problem* P, int j, double* o) {
  const int D = P->D, nv = 1 << D;
  const double hD = std::pow(P->h, D);
  double a[3], bb[3];
  P->cell_box(j, a, bb);
  for (int v = 0; v < nv; ++v) {
    double x[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) x[d] = (v >> d) & 1 ? bb[d] : a[d];
    o[v] = P->phi(x) / (P->h * P->h);
  }
  double fa = 0.0, fb = 0.0;
  const int pa = P->cellpart[2 * j], pb = P->cellpart[2 * j + 1];
  if (pa >= 0) fa = P->parts[pa].vol / hD;
  if (pb >= 0) fb = P->parts[pb].vol / hD;
  o[nv] = fa;
  o[nv + 1] = fb;
}

void xp_block_features(void* h, double* out) {
  Problem* P = static_cast<Problem*>(h);
  const Level& L = P->levels[0];
  const int nv = 1 << P->D;
  for (int b = 0; b < L.nb; ++b) cell_features(P, L.rep[b], out + (size_t)b * (nv + 2));
}

void xp_cell_features(void* h, int n, const int32_t* cells, double* out) {
  Problem* P = static_cast<Problem*>(h);
  const int nv = 1 << P->D;
  for (int i = 0; i < n; ++i) cell_features(P, cells[i], out + (size_t)i * (nv + 2));
}

int xp_cut_cells(void* h, int32_t* out) {
  Problem* P = static_cast<Problem*>(h);
  const Level& L = P->levels[0];
  int cnt = 0;
  for (int j = 0; j < P->ncell; ++j) {
    const int pa = P->cellpart[2 * j], pb = P->cellpart[2 * j + 1];
    if (pa < 0 || pb < 0) continue;
    if (out) {
      out[3 * cnt] = j;
      out[3 * cnt + 1] = L.part_block[pa];
      out[3 * cnt + 2] = L.part_block[pb];
    }
    ++cnt;
  }
  return cnt;
}

}  // extern "C"
