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
