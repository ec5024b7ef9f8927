/* Random sequential addition of hard spheres in a cubic periodic box.
 *
 * Input generator only (holds none of the PSE method's arithmetic).  Seeded
 * with splitmix64 -> xoshiro256** (public-domain generators by Vigna), so the
 * same seed gives the same configuration on every host.  Spheres of radius a are
 * proposed uniformly in [0, L)^3 and accepted when no centre lies closer than
 * 2a (minimum image); a linked-cell grid of side >= 2a makes each test O(1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
typedef struct { uint64_t s[4]; } rng_t;
static uint64_t splitmix(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t next(rng_t *r) {
  uint64_t *s = r->s, res = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t; s[3] = rotl(s[3], 45);
  return res;
}
static double unif(rng_t *r) { return (double)(next(r) >> 11) * 0x1.0p-53; }

/* Returns the number of placed spheres (== N on success). */
int64_t pse_rsa(int64_t N, double L, double a, uint64_t seed, int64_t max_attempts, double *pos) {
  rng_t r;
  uint64_t sm = seed;
  for (int i = 0; i < 4; ++i) r.s[i] = splitmix(&sm);
  int64_t nc = (int64_t)floor(L / (2.0 * a));
  if (nc < 1) nc = 1;
  if (nc > 1024) nc = 1024;
  double cs = L / (double)nc, d2min = 4.0 * a * a;
  int64_t ncell = nc * nc * nc;
  int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
  int64_t *nxt = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
  if (!head || !nxt) { free(head); free(nxt); return -1; }
  for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
  int64_t placed = 0;
  for (int64_t att = 0; att < max_attempts && placed < N; ++att) {
    double x[3] = {unif(&r) * L, unif(&r) * L, unif(&r) * L};
    int64_t ci[3];
    for (int d = 0; d < 3; ++d) { ci[d] = (int64_t)(x[d] / cs); if (ci[d] >= nc) ci[d] = nc - 1; }
    int ok = 1;
    int span = nc >= 3 ? 1 : 0;
    for (int dz = -span; dz <= span && ok; ++dz)
      for (int dy = -span; dy <= span && ok; ++dy)
        for (int dx = -span; dx <= span && ok; ++dx) {
          int64_t c = (((ci[2] + dz + nc) % nc) * nc + (ci[1] + dy + nc) % nc) * nc + (ci[0] + dx + nc) % nc;
          for (int64_t j = head[c]; j >= 0; j = nxt[j]) {
            double s2 = 0.0;
            for (int d = 0; d < 3; ++d) {
              double dd = x[d] - pos[3 * j + d];
              dd -= L * nearbyint(dd / L);
              s2 += dd * dd;
            }
            if (s2 < d2min) { ok = 0; break; }
          }
        }
    if (!ok && nc >= 3) continue;
    if (nc < 3) { /* tiny boxes: check all placed spheres */
      ok = 1;
      for (int64_t j = 0; j < placed && ok; ++j) {
        double s2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          double dd = x[d] - pos[3 * j + d];
          dd -= L * nearbyint(dd / L);
          s2 += dd * dd;
        }
        if (s2 < d2min) ok = 0;
      }
      if (!ok) continue;
    }
    int64_t c = (ci[2] * nc + ci[1]) * nc + ci[0];
    for (int d = 0; d < 3; ++d) pos[3 * placed + d] = x[d];
    nxt[placed] = head[c];
    head[c] = placed;
    ++placed;
  }
  free(head);
  free(nxt);
  return placed;
}

/* Dense hard-sphere configurations (phi above the RSA limit near 0.38):
 * uniform random centres at the target density, overlaps removed by repeated
 * pairwise push-apart passes (each overlapping pair is separated along its line
 * of centres to slightly beyond contact), then `sweeps` hard-sphere Monte Carlo
 * displacement sweeps (step adapted towards 40% acceptance) to randomise the
 * packing.  Returns 0 on success, -1 if overlaps remain after max_iter passes. */
static int64_t cell_of(const double *x, double cs, int64_t nc) {
  int64_t c[3];
  for (int d = 0; d < 3; ++d) {
    c[d] = (int64_t)(x[d] / cs);
    if (c[d] >= nc) c[d] = nc - 1;
    if (c[d] < 0) c[d] = 0;
  }
  return (c[2] * nc + c[1]) * nc + c[0];
}

static void build_cells(int64_t N, const double *pos, double cs, int64_t nc, int64_t *head, int64_t *nxt) {
  for (int64_t c = 0; c < nc * nc * nc; ++c) head[c] = -1;
  for (int64_t i = 0; i < N; ++i) {
    int64_t c = cell_of(pos + 3 * i, cs, nc);
    nxt[i] = head[c];
    head[c] = i;
  }
}

static double wrapd(double x, double L) {
  x = fmod(x, L);
  if (x < 0) x += L;
  if (x >= L) x = 0.0;
  return x;
}

int64_t pse_pack(int64_t N, double L, double a, uint64_t seed, int64_t sweeps, int64_t max_iter, double *pos) {
  rng_t r;
  uint64_t sm = seed;
  for (int i = 0; i < 4; ++i) r.s[i] = splitmix(&sm);
  double delta = 0.1 * a;
  int64_t nc = (int64_t)floor(L / (2.0 * a + 2.0 * sqrt(3.0) * delta));
  if (nc < 3) return -1;
  if (nc > 1024) nc = 1024;
  double cs = L / (double)nc, d2min = 4.0 * a * a;
  int64_t *head = (int64_t *)malloc(sizeof(int64_t) * nc * nc * nc);
  int64_t *nxt = (int64_t *)malloc(sizeof(int64_t) * N);
  double *disp = (double *)malloc(sizeof(double) * 3 * N);
  if (!head || !nxt || !disp) { free(head); free(nxt); free(disp); return -1; }
  for (int64_t i = 0; i < 3 * N; ++i) pos[i] = unif(&r) * L;
  int64_t it = 0, over = 1;
  for (; it < max_iter && over; ++it) {
    build_cells(N, pos, cs, nc, head, nxt);
    for (int64_t i = 0; i < 3 * N; ++i) disp[i] = 0.0;
    over = 0;
    for (int64_t i = 0; i < N; ++i) {
      int64_t ci = cell_of(pos + 3 * i, cs, nc), cz = ci / (nc * nc), cy = (ci / nc) % nc, cx = ci % nc;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int64_t c = (((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cx + dx + nc) % nc;
            for (int64_t j = head[c]; j >= 0; j = nxt[j]) {
              if (j <= i) continue;
              double d[3], s2 = 0.0;
              for (int k = 0; k < 3; ++k) {
                d[k] = pos[3 * i + k] - pos[3 * j + k];
                d[k] -= L * nearbyint(d[k] / L);
                s2 += d[k] * d[k];
              }
              if (s2 >= d2min) continue;
              ++over;
              double rr = sqrt(s2);
              if (rr < 1e-12) { d[0] = 1.0; d[1] = d[2] = 0.0; rr = 1.0; s2 = 0.0; }
              double push = 0.5 * (2.0 * a * (1.0 + 1e-3) - sqrt(s2)) / rr;
              for (int k = 0; k < 3; ++k) {
                disp[3 * i + k] += push * d[k];
                disp[3 * j + k] -= push * d[k];
              }
            }
          }
    }
    for (int64_t i = 0; i < 3 * N; ++i) pos[i] = wrapd(pos[i] + disp[i], L);
  }
  if (over) { free(head); free(nxt); free(disp); return -1; }
  /* hard-sphere Monte Carlo sweeps (cells of side >= 2a + 2 sqrt(3) delta, rebuilt per sweep) */
  for (int64_t sw = 0; sw < sweeps; ++sw) {
    build_cells(N, pos, cs, nc, head, nxt);
    int64_t acc = 0;
    for (int64_t i = 0; i < N; ++i) {
      double x[3];
      for (int k = 0; k < 3; ++k) x[k] = wrapd(pos[3 * i + k] + delta * (2.0 * unif(&r) - 1.0), L);
      int64_t ci = cell_of(pos + 3 * i, cs, nc), cz = ci / (nc * nc), cy = (ci / nc) % nc, cx = ci % nc;
      int ok = 1;
      for (int dz = -1; dz <= 1 && ok; ++dz)
        for (int dy = -1; dy <= 1 && ok; ++dy)
          for (int dx = -1; dx <= 1 && ok; ++dx) {
            int64_t c = (((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cx + dx + nc) % nc;
            for (int64_t j = head[c]; j >= 0 && ok; j = nxt[j]) {
              if (j == i) continue;
              double s2 = 0.0;
              for (int k = 0; k < 3; ++k) {
                double dd = x[k] - pos[3 * j + k];
                dd -= L * nearbyint(dd / L);
                s2 += dd * dd;
              }
              if (s2 < d2min) ok = 0;
            }
          }
      if (ok) {
        for (int k = 0; k < 3; ++k) pos[3 * i + k] = x[k];
        ++acc;
      }
    }
    double rate = (double)acc / (double)N, nd = delta * (rate > 0.4 ? 1.05 : 0.95);
    if (2.0 * a + 2.0 * sqrt(3.0) * nd <= cs) delta = nd;  /* keep the stale-cell search valid */
  }
  free(head);
  free(nxt);
  free(disp);
  return 0;
}
