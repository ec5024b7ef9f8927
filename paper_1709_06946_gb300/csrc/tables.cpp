// Host-side parameter rules, real-space mobility tables and small dense algebra.
//
// Real-space functions (Sec. 2.2: inverse Fourier transform of M - M^(w); App. A).
// The Fourier-space pair mobilities are the Hasimoto Green's function times
// shape factors; sin(ka)/ka is the transform of the unit sphere-shell density and
// 3 (sin ka - ka cos ka)/(ka)^3 that of the unit ball.  With the split Green's
// function J^(r) = (1/eta)[I phi0 + grad grad psi0], phi0 = FT^-1[(1-H)/k^2],
// psi0 = FT^-1[(1-H)/k^4], every block is a derivative of a shell/ball
// convolution of J^(r):
//   M_UF = T_aa,  M_UC_imn = -d_n T_ab_im,  M_DF_ijm = d_j T_ab_im,
//   M_DC_ijmn = -d_j d_n T_bb_im,  T_k = (1/eta)[I Phi_k + grad grad Psi_k].
// For radial functions the 3D convolution is a 1D convolution of the profiles
// t f(t) with an even piecewise-polynomial kernel w_k on [-2a, 2a]; the profile
// of psi0 splits into the Oseen part -t|t|/(8 pi) and an entire remainder, so
// each convolution is a piecewise-polynomial x smooth integral, done here by
// Gauss-Legendre quadrature between the kinks (plus the point masses that the
// Oseen part's higher derivatives carry).
//
// The seven tabulated scalars act on a pair with unit separation vector rh
// (rh = (x_alpha - x_beta)/r), source moments F, S (tensor) / s (Y components):
//   U = fperp F + (fpar - fperp)(rh.F) rh + gS (S rh) + gR (rh.S.rh) rh
//   e = -(gS/2) symY(F, rh) - gR (rh.F) y(rh) + kS s + kX symY(S rh, rh) + kR (rh.S.rh) y(rh)
// with symY(p, q) the Y components of p q^T + q p^T and y(rh) those of rh rh^T.
#include <algorithm>
#include <cmath>

#include "krylov_math.cuh"
#include "pse_internal.cuh"

namespace pse {
namespace {

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- parameter rules
double hasimoto(double u) { return (1.0 + u) * std::exp(-u); }  // H as a function of u = k^2/4xi^2

double kcut_rule(double xi, double tol) {
  double lo = 0.0, hi = 800.0;  // H decreases in u
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (hasimoto(mid) > tol) lo = mid; else hi = mid;
  }
  return 2.0 * xi * std::sqrt(hi);
}

// Smallest P meeting Eq. bound (C = 1, m = sqrt(pi P)) with the largest eigenvalue
// lam of A^T A of the lattice deformation (lam = 1: orthorhombic grids).
int support_rule(double tol, double lam) {
  for (int P = 1; P < 64; ++P) {
    double m = std::sqrt(kPi * P);
    double b = std::exp(-kPi * kPi * P * P / (2.0 * m * m * lam)) + std::erfc(m / std::sqrt(2.0 * lam));
    if (b <= tol) return P;
  }
  return 64;
}

// Eigenvalues of a symmetric 3 x 3 matrix (row-major) by cyclic Jacobi rotations.
void sym3_eigenvalues(const double S[9], double ev[3]) {
  double a[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) a[i][j] = S[3 * i + j];
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = std::fabs(a[0][1]) + std::fabs(a[0][2]) + std::fabs(a[1][2]);
    if (off < 1e-300) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        const double th = 0.5 * (a[q][q] - a[p][p]) / a[p][q];
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < 3; ++k) {  // columns p, q
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - sn * akq;
          a[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // rows p, q
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - sn * aqk;
          a[q][k] = sn * apk + c * aqk;
        }
      }
  }
  for (int i = 0; i < 3; ++i) ev[i] = a[i][i];
}

bool smooth2357(int n) {
  for (int f : {2, 3, 5, 7})
    while (n % f == 0) n /= f;
  return n == 1;
}

int next_grid(double x) {
  int n = std::max(2, (int)std::ceil(x - 1e-9));
  while (n % 2 || !smooth2357(n)) ++n;
  return n;
}

bool smooth23(int n) {
  for (int f : {2, 3})
    while (n % f == 0) n /= f;
  return n == 1;
}

// smallest even 2^i 3^j >= n
int ladder_grid(int n) {
  while (n % 2 || !smooth23(n)) ++n;
  return n;
}

// Padded row length (points) of a spreading tile; the kernels use the same rule.
int tile_row(int Tx, int P) {
  if (Tx >= 16) return Tx + (((P - Tx) % 8) + 8) % 8;
  return Tx + ((Tx & 3) == 0 ? 2 : 0);
}

int pick_tile(int Ng, int minsize, int cap, bool prefer8) {
  int best = -1;
  for (int d = 1; d <= Ng; ++d) {
    if (Ng % d || d < minsize || d > cap) continue;
    if (best < 0) { best = d; continue; }
    bool b8 = (best % 8) == 0, d8 = (d % 8) == 0;
    if (prefer8 && d8 != b8) { if (d8) best = d; continue; }
    if (d > best) best = d;
  }
  if (best < 0) {  // no divisor in range: smallest divisor >= minsize, else the whole side
    for (int d = minsize; d <= Ng; ++d)
      if (Ng % d == 0) { best = d; break; }
    if (best < 0) best = Ng;
  }
  return best;
}

// ---------------------------------------------------------------- Gauss-Legendre
struct GL {
  std::vector<double> x, w;
  explicit GL(int n) : x(n), w(n) {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

// 1D kernels w_k(s), even with support |s| <= 2a, unit integral:
//   shell*shell: (2a - |s|)/(4a^2)
//   shell*ball : (4a^3 - 3a s^2 + |s|^3)/(8a^4)
//   ball*ball  : 3 (32a^5 - 40a^3 s^2 + 20a^2 |s|^3 - |s|^5)/(160 a^6)
double wk(int k, double s, double a) {
  double t = std::fabs(s);
  if (t > 2.0 * a) return 0.0;
  if (k == 0) return (2.0 * a - t) / (4.0 * a * a);
  if (k == 1) return (4.0 * a * a * a - 3.0 * a * t * t + t * t * t) / (8.0 * a * a * a * a);
  double a3 = a * a * a;
  return 3.0 * (32.0 * a3 * a * a - 40.0 * a3 * t * t + 20.0 * a * a * t * t * t - t * t * t * t * t) /
         (160.0 * a3 * a3);
}
// d/ds and d2/ds2 of w_k for s > 0 (right limits at the breakpoints)
double wk_d1(int k, double s, double a) {
  if (s >= 2.0 * a) return 0.0;
  if (k == 0) return -1.0 / (4.0 * a * a);
  if (k == 1) return (-6.0 * a * s + 3.0 * s * s) / (8.0 * a * a * a * a);
  double a3 = a * a * a;
  return 3.0 * (-80.0 * a3 * s + 60.0 * a * a * s * s - 5.0 * s * s * s * s) / (160.0 * a3 * a3);
}
double wk_d2(int k, double s, double a) {
  if (s >= 2.0 * a) return 0.0;
  if (k == 0) return 0.0;
  if (k == 1) return (-6.0 * a + 6.0 * s) / (8.0 * a * a * a * a);
  double a3 = a * a * a;
  return 3.0 * (-80.0 * a3 + 120.0 * a * a * s - 20.0 * s * s * s) / (160.0 * a3 * a3);
}

// n-th derivative of the entire part of the profile t psi0(t):
//   (1/8pi) [t^2 erf(xi t) + t exp(-xi^2 t^2)/(xi sqrt(pi))]
double prof_smooth(int n, double t, double xi) {
  const double c = 1.0 / (8.0 * kPi), sp = std::sqrt(kPi);
  double E = std::erf(xi * t), g = std::exp(-xi * xi * t * t), u = xi * xi * t * t;
  switch (n) {
    case 0: return c * (t * t * E + t * g / (xi * sp));
    case 1: return c * (2.0 * t * E + g / (xi * sp));
    case 2: return c * (2.0 * E + 2.0 * xi / sp * t * g);
    case 3: return c * 2.0 * xi / sp * g * (3.0 - 2.0 * u);
    case 4: return c * 4.0 * xi * xi * xi / sp * t * g * (2.0 * u - 5.0);
    default: return c * 4.0 * xi * xi * xi / sp * g * (-4.0 * u * u + 16.0 * u - 5.0);
  }
}
// regular part of the n-th derivative of the Oseen profile -t|t|/(8 pi) (n <= 2)
double prof_free(int n, double t) {
  const double c = 1.0 / (8.0 * kPi);
  if (n == 0) return -c * t * std::fabs(t);
  if (n == 1) return -2.0 * c * std::fabs(t);
  if (n == 2) return t > 0 ? -2.0 * c : (t < 0 ? 2.0 * c : 0.0);
  return 0.0;
}

// Q_k^(n)(r) = int w_k(s) u^(n)(r - s) ds, r >= 0.
double conv(const GL &gl, int k, int n, double r, double xi, double a) {
  double rb = std::min(r, 2.0 * a);
  double edges[4] = {-2.0 * a, 0.0, rb, 2.0 * a};
  double sum = 0.0;
  for (int piece = 0; piece < 3; ++piece) {
    double lo = edges[piece], hi = edges[piece + 1];
    if (hi <= lo) continue;
    double hw = 0.5 * (hi - lo), mid = 0.5 * (hi + lo), acc = 0.0;
    for (size_t q = 0; q < gl.x.size(); ++q) {
      double s = mid + hw * gl.x[q], t = r - s;
      double f = prof_smooth(n, t, xi) + (n <= 2 ? prof_free(n, t) : 0.0);
      acc += gl.w[q] * wk(k, s, a) * f;
    }
    sum += hw * acc;
  }
  const double c4 = 4.0 / (8.0 * kPi);  // point masses: u''' = -4c delta, u'''' = -4c delta', ...
  if (n == 3) sum -= c4 * wk(k, r, a);
  if (n == 4) sum -= c4 * wk_d1(k, r, a);
  if (n == 5) sum -= c4 * wk_d2(k, r, a);
  return sum;
}

}  // namespace

int lattice_of(const double A[9], double Ai[9], double &det, double &lam_min, double &lam_max, double &cmax,
               std::string &err) {
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(A[i])) {
      err = "lattice deformation has a non-finite entry";
      return 1;
    }
  det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(det > 1e-12)) {
    err = "lattice deformation needs det A > 0";
    return 1;
  }
  // inverse by cofactors
  Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  double G[9], ev[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[3 * i + j] = A[i] * A[j] + A[3 + i] * A[3 + j] + A[6 + i] * A[6 + j];
  sym3_eigenvalues(G, ev);
  lam_min = std::min(ev[0], std::min(ev[1], ev[2]));
  lam_max = std::max(ev[0], std::max(ev[1], ev[2]));
  cmax = 0;
  for (int j = 0; j < 3; ++j) cmax = std::max(cmax, std::sqrt(G[4 * j]));
  return 0;
}

int set_lattice(Params &p, const double A[9], std::string &err) {
  double Ai[9], det, lmin, lmax, cm;
  if (lattice_of(A, Ai, det, lmin, lmax, cm, err)) return 1;
  bool ident = true;
  for (int i = 0; i < 9; ++i) ident = ident && A[i] == ((i % 4 == 0) ? 1.0 : 0.0);
  p.def = ident ? 0 : 1;
  for (int i = 0; i < 9; ++i) {
    p.A[i] = A[i];
    p.Ai[i] = Ai[i];
  }
  p.detA = det;
  p.lam_min = lmin;
  p.lam_max = lmax;
  p.cmax = cm;
  return 0;
}

int choose_params(Params &p, const pse_options &opt, std::string &err) {
  if (!(p.N >= 1) || !(p.L > 0) || !(p.a > 0) || !(p.eta > 0) || !(p.kT >= 0) || !(p.xi > 0) ||
      !(p.tol > 0 && p.tol <= 0.1)) {
    err = "invalid physical parameter (need N>=1, L,a,eta,xi>0, kT>=0, 0<tol<=0.1)";
    return 1;
  }
  p.rule = opt.rule;
  {  // lattice deformation (Sec. 2.3.3); all zero = the cube
    bool any = false;
    for (int i = 0; i < 9; ++i) any = any || opt.deform[i] != 0.0;
    const double I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (set_lattice(p, any ? opt.deform : I3, err)) return 1;
    p.lam_P = (p.def && opt.lambda_support) ? p.lam_max : 1.0;
    p.lam_cells = p.lam_min;
    p.cmax_grid = p.cmax;
  }
  double tq = p.rule == PSE_RULE_PAPER ? p.tol : p.tol / 10.0;
  p.rcut = opt.rcut > 0 ? opt.rcut
                        : (p.rule == PSE_RULE_PAPER ? std::sqrt(std::log(1.0 / p.tol)) / p.xi
                                                    : p.a + std::sqrt(std::log(10.0 / p.tol)) / p.xi);
  p.kcut = kcut_rule(p.xi, p.tol);
  p.P = opt.P > 0 ? opt.P : support_rule(tq, p.lam_P);
  p.m = std::sqrt(kPi * p.P);
  if (opt.Ng > 0) {
    p.Ng = opt.Ng;
  } else {
    p.Ng = next_grid(p.kcut * p.L * p.cmax / kPi);  // every |k| <= k_cut on the grid (cmax = 1 for the cube)
    while (true) {
      double h = p.L / p.Ng, eg = (h * p.P * p.xi / p.m) * (h * p.P * p.xi / p.m);
      if (eg < 1.0) break;
      p.Ng = next_grid(p.Ng + 1);
    }
    if (opt.grid_ladder) p.Ng = ladder_grid(p.Ng);  // a finer grid only lowers the NUFFT error
  }
  // half-width of the cell: L/2 for the cube, L sqrt(lambda_min)/2 on a deformed lattice
  const double half = 0.5 * p.L * std::sqrt(p.lam_cells);
  if (p.rcut > half * (1.0 + 1e-12)) {
    err = "r_cut " + std::to_string(p.rcut) + " exceeds the half-width " + std::to_string(half) +
          " of the cell (minimum-image pair sum): enlarge the box or increase xi";
    return 1;
  }
  // linked cells of side >= r_cut/2, searched with a 5 x 5 x 5 stencil (all cells when nc < 5); on a
  // deformed lattice the cells are cubes in lattice coordinates, where a pair closer than r_cut is
  // closer than r_cut / sqrt(lambda_min)
  p.nc = std::max(1, std::min(1023, (int)std::floor(2.0 * p.L * std::sqrt(p.lam_cells) / p.rcut)));
  p.cs = p.L / p.nc;
  const int caps[3] = {16, 16, 16};
  // The spreading tile must hold P - 1 points per side and fit shared memory; a
  // large support (deformed lattices) may need a grid with a suitable divisor: the
  // next 2,3,5,7-smooth sizes are tried (a finer grid only lowers the NUFFT error).
  for (int attempt = 0;; ++attempt) {
    p.h = p.L / p.Ng;
    p.eta_g = (p.h * p.P * p.xi / p.m) * (p.h * p.P * p.xi / p.m);
    p.nkx = p.Ng / 2 + 1;
    if (p.Ng % 2 || p.Ng < 4 || p.Ng > 4096) { err = "grid size must be even, 4..4096"; return 1; }
    if (p.P < 1 || p.P > 32 || p.P > p.Ng) { err = "support size out of range"; return 1; }
    if (!(p.eta_g < 1.0)) { err = "Gaussian width eta_g >= 1 (refine the grid)"; return 1; }
    std::string terr;
    if (choose_tile(p, caps, opt.tile, terr) == 0) return 0;
    if (opt.Ng > 0 || attempt >= 64) {
      err = terr;
      return 1;
    }
    p.Ng = next_grid(p.Ng + 1);
  }
}

// Spreading tile of a suspension: the largest divisors of Ng within caps (x
// prefers multiples of 8 for coalesced rows), shrunk until the CTA's shared
// memory fits the budget; fixed[d] > 0 overrides dimension d.
int choose_tile(Params &p, const int caps[3], const int fixed[3], std::string &err) {
  int mins = std::max(1, p.P - 1);
  // z planes are owned by the 16 warps of a spreading CTA: aim for 16 planes, x rows of up
  // to 16 points (coalesced stores), y up to the cap
  p.tile[0] = fixed[0] > 0 ? fixed[0] : pick_tile(p.Ng, mins, caps[0], true);
  p.tile[1] = fixed[1] > 0 ? fixed[1] : pick_tile(p.Ng, mins, caps[1], false);
  p.tile[2] = fixed[2] > 0 ? fixed[2] : pick_tile(p.Ng, mins, caps[2], false);
  // shared memory of a spreading/interpolation CTA with 8 components (the
  // largest): the tile with its padded rows; the 8-component kernels then run
  // one CTA per SM and the 5-component ones (the GMRES loop) two
  auto smem = [&]() { return (size_t)8 * p.tile[2] * p.tile[1] * tile_row(p.tile[0], p.P) * p.ts; };
  const size_t budget = 200 * 1024;
  while (smem() > budget) {  // shrink the larger of x and y first, z last
    const int order[3] = {p.tile[0] >= p.tile[1] ? 0 : 1, p.tile[0] >= p.tile[1] ? 1 : 0, 2};
    bool shrunk = false;
    for (int d : order) {
      if (fixed[d] > 0) continue;
      const int nt = pick_tile(p.Ng, mins, p.tile[d] - 1, d == 0);
      if (nt < p.tile[d]) {
        p.tile[d] = nt;
        shrunk = true;
        break;
      }
    }
    if (!shrunk) break;
  }
  if (smem() > 220 * 1024) {  // the opt-in limit is 227 KB less the kernels' static shared memory
    err = "spreading tile exceeds the shared-memory limit; choose a smaller tile";
    return 1;
  }
  for (int d = 0; d < 3; ++d) {
    if (p.Ng % p.tile[d] || (p.tile[d] < p.P - 1 && p.tile[d] != p.Ng)) {
      err = "tile sizes must divide Ng and be >= P-1";
      return 1;
    }
    if (p.tile[d] > 256) {  // the kernels pack tile offsets into 10-bit fields
      err = "tile sizes must be at most 256";
      return 1;
    }
    p.ntile[d] = p.Ng / p.tile[d];
  }
  return 0;
}

void real_functions(const Params &p, double r, double out[7]) {
  static const GL gl(40);
  double a = p.a, xi = p.xi, eta = p.eta;
  double Q[3][5];
  for (int k = 0; k < 3; ++k)
    for (int n = 0; n < 5; ++n) Q[k][n] = conv(gl, k, n, r, xi, a);
  double r2 = r * r, r3 = r2 * r, r4 = r3 * r, r5 = r4 * r;
  double Phi[3][3], Psi[3][5];
  for (int k = 0; k < 3; ++k) {
    const double *U = Q[k];
    Psi[k][1] = U[1] / r - U[0] / r2;
    Psi[k][2] = U[2] / r - 2 * U[1] / r2 + 2 * U[0] / r3;
    Psi[k][3] = U[3] / r - 3 * U[2] / r2 + 6 * U[1] / r3 - 6 * U[0] / r4;
    Psi[k][4] = U[4] / r - 4 * U[3] / r2 + 12 * U[2] / r3 - 24 * U[1] / r4 + 24 * U[0] / r5;
    double V0 = -U[2], V1 = -U[3], V2 = -U[4];  // r Phi = -U''  (lap psi0 = -phi0)
    Phi[k][0] = V0 / r;
    Phi[k][1] = V1 / r - V0 / r2;
    Phi[k][2] = V2 / r - 2 * V1 / r2 + 2 * V0 / r3;
  }
  auto Ap = [&](int k) { return Psi[k][2] / r - Psi[k][1] / r2; };
  auto D = [&](int k) { return Psi[k][3] - 3 * Psi[k][2] / r + 3 * Psi[k][1] / r2; };
  auto Dp = [&](int k) {
    return Psi[k][4] - 3 * Psi[k][3] / r + 6 * Psi[k][2] / r2 - 6 * Psi[k][1] / r3;
  };
  out[0] = (Phi[0][0] + Psi[0][1] / r) / eta;                           // fperp
  out[1] = (Phi[0][0] + Psi[0][2]) / eta;                               // fpar
  out[2] = -(Phi[1][1] + 2 * Ap(1)) / eta;                              // gS
  out[3] = -D(1) / eta;                                                 // gR
  out[4] = -(Phi[2][1] / r + 2 * Ap(2) / r) / eta;                      // kS
  out[5] = -(0.5 * (Phi[2][2] - Phi[2][1] / r) + 2 * D(2) / r) / eta;   // kX
  out[6] = -(Dp(2) - 3 * D(2) / r) / eta;                               // kR
}

void rot_functions(const Params &p, double r, double out[3]) {
  static const GL gl(40);
  const double a = p.a, xi = p.xi, eta = p.eta;
  // Phi = V/r, V = -U'' for the shell*ball (k = 1) and ball*ball (k = 2) convolutions
  double U[3][5];
  for (int k = 1; k < 3; ++k)
    for (int n = 2; n < 5; ++n) U[k][n] = conv(gl, k, n, r, xi, a);
  const double r2 = r * r, r3 = r2 * r;
  double Phi1[3], Phi2[3];
  for (int k = 1; k < 3; ++k) {
    const double V0 = -U[k][2], V1 = -U[k][3], V2 = -U[k][4];
    Phi1[k] = V1 / r - V0 / r2;
    Phi2[k] = V2 / r - 2 * V1 / r2 + 2 * V0 / r3;
  }
  out[0] = Phi1[1] / (2 * eta);
  out[1] = -(Phi2[2] + Phi1[2] / r) / (4 * eta);
  out[2] = (Phi2[2] - Phi1[2] / r) / (4 * eta);
}

void build_rot_table(const Params &p, int points_per_2a, int len, std::vector<double> &v, double *self_ol) {
  static const GL gl(40);
  const double dr = 2.0 * p.a / points_per_2a;
  const double sol = conv(gl, 2, 5, 0.0, p.xi, p.a) / (6.0 * p.eta);
  v.assign((size_t)len * 4, 0.0);
  const double z[3] = {0.0, sol, 0.0};
  const int ismall = (int)std::ceil(0.05 * p.a / dr);
  double f[3], fs[3] = {0, 0, 0};
  rot_functions(p, ismall * dr, fs);
  for (int i = 0; i < len; ++i) {
    if (i == 0) {
      for (int q = 0; q < 3; ++q) f[q] = z[q];
    } else if (i < ismall) {  // below 0.05a the formulas cancel badly: interpolate to the r -> 0 limit
      const double w = (double)i / ismall;
      for (int q = 0; q < 3; ++q) f[q] = (1 - w) * z[q] + w * fs[q];
    } else {
      rot_functions(p, i * dr, f);
    }
    for (int q = 0; q < 3; ++q) v[(size_t)i * 4 + q] = f[q];
  }
  *self_ol = sol;
}

void build_real_table(const Params &p, int points_per_2a, RealTable &t) {
  static const GL gl(40);
  t.dr = 2.0 * p.a / points_per_2a;
  t.k2 = points_per_2a;
  t.len = (int)std::ceil(p.rcut / t.dr) + 4;
  t.v.assign((size_t)t.len * 8, 0.0);
  // self terms: UF = (2/3) Phi_aa(0)/eta with Phi(0) = -U'''(0); ES = U_bb^(5)(0)/(5 eta)
  t.self_uf = (2.0 / 3.0) * (-conv(gl, 0, 3, 0.0, p.xi, p.a)) / p.eta;
  t.self_es = conv(gl, 2, 5, 0.0, p.xi, p.a) / (5.0 * p.eta);
  double rsmall = 0.05 * p.a;
  int ismall = (int)std::ceil(rsmall / t.dr);
  double f[7];
  for (int i = 1; i < t.len; ++i) {
    double r = std::max(i, ismall) * t.dr;
    real_functions(p, r, f);
    for (int q = 0; q < 7; ++q) t.v[(size_t)i * 8 + q] = f[q];
  }
  double z[7] = {t.self_uf, t.self_uf, 0.0, 0.0, t.self_es, 0.0, 0.0};
  for (int q = 0; q < 7; ++q) t.v[q] = z[q];
  // below 0.05a the formulas cancel badly: interpolate linearly to the r -> 0 limit
  for (int i = 1; i < ismall; ++i) {
    double w = (double)i / ismall;
    for (int q = 0; q < 7; ++q) t.v[(size_t)i * 8 + q] = (1 - w) * z[q] + w * t.v[(size_t)ismall * 8 + q];
  }
}

void fill_real_table_f32(const Params &p, int points_per_2a, int len, float *out, double *self_uf,
                         double *self_es) {
  static const GL gl(40);
  double dr = 2.0 * p.a / points_per_2a;
  double suf = (2.0 / 3.0) * (-conv(gl, 0, 3, 0.0, p.xi, p.a)) / p.eta;
  double ses = conv(gl, 2, 5, 0.0, p.xi, p.a) / (5.0 * p.eta);
  int ismall = (int)std::ceil(0.05 * p.a / dr);
  double f[7], fs[7] = {0, 0, 0, 0, 0, 0, 0};
  const double z[7] = {suf, suf, 0.0, 0.0, ses, 0.0, 0.0};
  for (int i = len - 1; i >= 0; --i) {
    if (i == 0) {
      for (int q = 0; q < 7; ++q) f[q] = z[q];
    } else if (i < ismall) {
      double w = (double)i / ismall;
      for (int q = 0; q < 7; ++q) f[q] = (1 - w) * z[q] + w * fs[q];
    } else {
      real_functions(p, i * dr, f);
      if (i == ismall)
        for (int q = 0; q < 7; ++q) fs[q] = f[q];
    }
    for (int q = 0; q < 7; ++q) out[(size_t)i * 8 + q] = (float)f[q];
    out[(size_t)i * 8 + 7] = 0.0f;
  }
  *self_uf = suf;
  *self_es = ses;
}

bool tridiag_eigen(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &Z) {
  Z.assign((size_t)n * n, 0.0);
  e.resize(n, 0.0);
  return tql_eigen(n, d.data(), e.data(), Z.data());
}

}  // namespace pse

// ------------------------------------------------------------------ host test hooks
extern "C" {
// Seven real-space scalars at separations r[0..n) for the given physical parameters
// (out: n x 7); returns the self terms in self2[0..2).  Host only.
int pse_internal_real_functions(double a, double eta, double xi, int n, const double *r, double *out,
                                double *self2) {
  pse::Params p{};
  p.a = a;
  p.eta = eta;
  p.xi = xi;
  for (int i = 0; i < n; ++i) pse::real_functions(p, r[i], out + 7 * (size_t)i);
  if (self2) {
    pse::RealTable t;
    p.rcut = 2.0 * a;
    pse::build_real_table(p, 16, t);
    self2[0] = t.self_uf;
    self2[1] = t.self_es;
  }
  return 0;
}

// Spreading tile for a grid of Ng points per side, support P and real size ts
// (4 or 8 bytes) under the caps (fixed > 0 forces a side); tile and padded row
// length in out[0..4) (x, y, z, row).  Returns 0, or 1 when no tile fits.
int pse_internal_choose_tile(int Ng, int P, int ts, const int *caps, const int *fixed, int *out) {
  pse::Params p{};
  p.Ng = Ng;
  p.P = P;
  p.ts = ts;
  std::string err;
  if (pse::choose_tile(p, caps, fixed, err)) return 1;
  for (int d = 0; d < 3; ++d) out[d] = p.tile[d];
  out[3] = pse::tile_row(p.tile[0], P);
  return 0;
}

// c = T^{1/2} e_1 for the symmetric tridiagonal T (diagonal d, off-diagonal e).
int pse_internal_tridiag_sqrt_e1(int n, const double *d, const double *e, double *c) {
  std::vector<double> dd(d, d + n), ee(e, e + (n > 1 ? n - 1 : 0)), Z;
  if (!pse::tridiag_eigen(n, dd, ee, Z)) return 1;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += Z[(size_t)i * n + k] * std::sqrt(std::max(dd[k], 0.0)) * Z[k];
    c[i] = s;
  }
  return 0;
}
}
