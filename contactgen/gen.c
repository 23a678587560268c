/*
 * Seeded synthetic two-block contact problems (input generator only).
 *
 * This module produces the INPUTS of the interior-point Newton system
 * (K, J, D, b of the statically condensed system A u = b, Section 3,
 * eq. (linsystem1)).  It holds none of the solver's arithmetic: no Schur
 * complement, no AMG, no filter, no Krylov method.  Both the CPU oracle and
 * the GPU library consume what it writes.
 *
 * Geometry (stand-in for the two-block problem of Section 4 / Section 6.1):
 *   lower block [0,1]x[0,1]x[0,1/2], upper block [0,1]x[0,1]x[1/2,1],
 *   each meshed by nx*ny*nz trilinear (Q1) hexahedra, with separate node sets
 *   that coincide on the interface z = 1/2.
 * Material: isotropic linear elasticity, sigma = lambda div(u) I + 2 mu eps(u)
 *   (Section 2.2), E and nu given, Lame parameters derived from them.
 * Element stiffness: 2x2x2 Gauss quadrature (exact for the affine brick).
 * Dirichlet: lower block bottom face and (optionally) upper block top face are
 *   clamped; clamped nodes are eliminated from the numbering.
 * Numbering: free nodes lexicographic with x fastest, then y, then z; lower
 *   block first.  DOF = 3*node + component (x, y, z interleaved).
 * Contact: node-to-node normal contact, one constraint per interface node pair
 *   (i, j): row r = j*(nx+1) + i of J carries -1 at the lower node's u_z and
 *   +1 at the upper node's u_z (linearised gap J u + g >= 0, Section 2.2).
 * Barrier diagonal D_r = 10^U(lo, hi) and right-hand side b_k ~ N(0, 1), drawn
 *   in that order from xoshiro256** (Blackman & Vigna) seeded through
 *   SplitMix64; uniforms from the top 53 bits; normals by Box-Muller.
 *
 * Plain C99 + optional OpenMP; compiled with -ffp-contract=off so that x86 and
 * Arm hosts produce the same matrices.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nx, ny, nz;          /* elements per block in x, y, z */
  int clamp_bottom;        /* clamp lower block z = 0 face */
  int clamp_top;           /* clamp upper block z = 1 face */
  double E, nu;            /* Young modulus, Poisson ratio */
} cg_geom;

/* ---------------- numbering ---------------- */

static int64_t layers_lower(const cg_geom* g) { return g->nz + 1 - (g->clamp_bottom ? 1 : 0); }
static int64_t layers_upper(const cg_geom* g) { return g->nz + 1 - (g->clamp_top ? 1 : 0); }
static int64_t plane(const cg_geom* g) { return (int64_t)(g->nx + 1) * (g->ny + 1); }

/* free-node index of grid node (i,j,k) of block `blk` (0 lower, 1 upper), or -1 if clamped */
static int64_t node_index(const cg_geom* g, int blk, int i, int j, int k) {
  int64_t kk;
  if (blk == 0) {
    if (g->clamp_bottom && k == 0) return -1;
    kk = k - (g->clamp_bottom ? 1 : 0);
    return (kk * (g->ny + 1) + j) * (int64_t)(g->nx + 1) + i;
  } else {
    if (g->clamp_top && k == g->nz) return -1;
    kk = k;
    return layers_lower(g) * plane(g) + (kk * (g->ny + 1) + j) * (int64_t)(g->nx + 1) + i;
  }
}

int64_t cg_num_nodes(const cg_geom* g) { return (layers_lower(g) + layers_upper(g)) * plane(g); }
int64_t cg_num_dofs(const cg_geom* g) { return 3 * cg_num_nodes(g); }
int64_t cg_num_constraints(const cg_geom* g) { return plane(g); }

/* node -> (blk, i, j, k) */
static void node_coords(const cg_geom* g, int64_t node, int* blk, int* i, int* j, int* k) {
  int64_t nl = layers_lower(g) * plane(g);
  int64_t loc;
  if (node < nl) { *blk = 0; loc = node; } else { *blk = 1; loc = node - nl; }
  *i = (int)(loc % (g->nx + 1));
  loc /= (g->nx + 1);
  *j = (int)(loc % (g->ny + 1));
  loc /= (g->ny + 1);
  *k = (int)loc + ((*blk == 0 && g->clamp_bottom) ? 1 : 0);
}

/* ---------------- element stiffness ---------------- */

/* Q1 brick of size hx*hy*hz; local node a = ax + 2 ay + 4 az.
 * Ke[(a*3+c)*24 + (b*3+d)] = int  lambda d_c phi_a d_d phi_b
 *                              + mu d_d phi_a d_c phi_b
 *                              + mu delta_cd grad phi_a . grad phi_b          */
void cg_element_stiffness(double hx, double hy, double hz, double E, double nu, double* Ke) {
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  const double gp = 1.0 / sqrt(3.0);
  const double h[3] = {hx, hy, hz};
  memset(Ke, 0, sizeof(double) * 24 * 24);
  for (int q = 0; q < 8; ++q) {
    const double xi[3] = {(q & 1) ? gp : -gp, (q & 2) ? gp : -gp, (q & 4) ? gp : -gp};
    const double detJ = (hx * 0.5) * (hy * 0.5) * (hz * 0.5);
    double grad[8][3];
    for (int a = 0; a < 8; ++a) {
      const double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
      const double f[3] = {1.0 + s[0] * xi[0], 1.0 + s[1] * xi[1], 1.0 + s[2] * xi[2]};
      for (int c = 0; c < 3; ++c) {
        double v = s[c] / 8.0;
        for (int e = 0; e < 3; ++e)
          if (e != c) v *= f[e];
        grad[a][c] = v * (2.0 / h[c]);
      }
    }
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) {
        double gg = grad[a][0] * grad[b][0] + grad[a][1] * grad[b][1] + grad[a][2] * grad[b][2];
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) {
            double v = lam * grad[a][c] * grad[b][d] + mu * grad[a][d] * grad[b][c];
            if (c == d) v += mu * gg;
            Ke[(a * 3 + c) * 24 + (b * 3 + d)] += detJ * v;
          }
      }
  }
  /* make the rounding symmetric: K is assembled from Ke, and an exactly
     symmetric K keeps every downstream operator exactly symmetric */
  for (int r = 0; r < 24; ++r)
    for (int c = r + 1; c < 24; ++c) {
      double v = 0.5 * (Ke[r * 24 + c] + Ke[c * 24 + r]);
      Ke[r * 24 + c] = v;
      Ke[c * 24 + r] = v;
    }
}

/* ---------------- stiffness assembly (CSR, rows in ascending column order) ---------------- */

/* number of free neighbour nodes (incl. itself) of a node */
static int count_neighbours(const cg_geom* g, int blk, int i, int j, int k) {
  int cnt = 0;
  for (int dk = -1; dk <= 1; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        int ii = i + di, jj = j + dj, kk = k + dk;
        if (ii < 0 || ii > g->nx || jj < 0 || jj > g->ny || kk < 0 || kk > g->nz) continue;
        if (node_index(g, blk, ii, jj, kk) < 0) continue;
        cnt++;
      }
  return cnt;
}

/* Fill row_ptr (length n+1) of K. */
int64_t cg_K_rowptr(const cg_geom* g, int64_t* row_ptr) {
  const int64_t nn = cg_num_nodes(g);
  row_ptr[0] = 0;
  /* per-node counts first (parallel), then prefix sum (serial) */
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < nn; ++p) {
    int blk, i, j, k;
    node_coords(g, p, &blk, &i, &j, &k);
    int c = count_neighbours(g, blk, i, j, k) * 3;
    row_ptr[3 * p + 1] = c;
    row_ptr[3 * p + 2] = c;
    row_ptr[3 * p + 3] = c;
  }
  for (int64_t r = 0; r < 3 * nn; ++r) row_ptr[r + 1] += row_ptr[r];
  return row_ptr[3 * nn];
}

/* Fill col_idx / val of K given row_ptr from cg_K_rowptr. */
void cg_K_fill(const cg_geom* g, const int64_t* row_ptr, int32_t* col_idx, double* val) {
  const int64_t nn = cg_num_nodes(g);
  const double hx = 1.0 / g->nx, hy = 1.0 / g->ny, hz = 0.5 / g->nz;
  double Ke[24 * 24];
  cg_element_stiffness(hx, hy, hz, g->E, g->nu, Ke);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < nn; ++p) {
    int blk, i, j, k;
    node_coords(g, p, &blk, &i, &j, &k);
    int64_t pos[3] = {row_ptr[3 * p], row_ptr[3 * p + 1], row_ptr[3 * p + 2]};
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          int ii = i + di, jj = j + dj, kk = k + dk;
          if (ii < 0 || ii > g->nx || jj < 0 || jj > g->ny || kk < 0 || kk > g->nz) continue;
          int64_t q = node_index(g, blk, ii, jj, kk);
          if (q < 0) continue;
          double blkv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          /* elements containing both p and q */
          for (int ck = k - 1; ck <= k; ++ck) {
            if (ck < 0 || ck >= g->nz || kk - ck < 0 || kk - ck > 1) continue;
            for (int cj = j - 1; cj <= j; ++cj) {
              if (cj < 0 || cj >= g->ny || jj - cj < 0 || jj - cj > 1) continue;
              for (int ci = i - 1; ci <= i; ++ci) {
                if (ci < 0 || ci >= g->nx || ii - ci < 0 || ii - ci > 1) continue;
                int la = (i - ci) + 2 * (j - cj) + 4 * (k - ck);
                int lb = (ii - ci) + 2 * (jj - cj) + 4 * (kk - ck);
                for (int c = 0; c < 3; ++c)
                  for (int d = 0; d < 3; ++d) blkv[c * 3 + d] += Ke[(la * 3 + c) * 24 + (lb * 3 + d)];
              }
            }
          }
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) {
              col_idx[pos[c]] = (int32_t)(3 * q + d);
              val[pos[c]] = blkv[c * 3 + d];
              pos[c]++;
            }
        }
  }
}

/* ---------------- contact Jacobian ---------------- */

/* J: m x n CSR, 2 entries per row; returns nnz. row_ptr length m+1. */
int64_t cg_J_fill(const cg_geom* g, int64_t* row_ptr, int32_t* col_idx, double* val) {
  const int64_t m = cg_num_constraints(g);
  for (int j = 0; j <= g->ny; ++j)
    for (int i = 0; i <= g->nx; ++i) {
      int64_t r = (int64_t)j * (g->nx + 1) + i;
      int64_t lo = node_index(g, 0, i, j, g->nz);
      int64_t up = node_index(g, 1, i, j, 0);
      row_ptr[r] = 2 * r;
      /* ascending column order: lower block nodes precede upper block nodes */
      col_idx[2 * r] = (int32_t)(3 * lo + 2);
      val[2 * r] = -1.0;
      col_idx[2 * r + 1] = (int32_t)(3 * up + 2);
      val[2 * r + 1] = 1.0;
    }
  row_ptr[m] = 2 * m;
  return 2 * m;
}

/* nodal coordinates (for tests: rigid-body modes, patch tests); xyz length 3*nodes */
void cg_node_xyz(const cg_geom* g, double* xyz) {
  const int64_t nn = cg_num_nodes(g);
  for (int64_t p = 0; p < nn; ++p) {
    int blk, i, j, k;
    node_coords(g, p, &blk, &i, &j, &k);
    xyz[3 * p + 0] = (double)i / g->nx;
    xyz[3 * p + 1] = (double)j / g->ny;
    xyz[3 * p + 2] = 0.5 * blk + 0.5 * (double)k / g->nz;
  }
}

/* ---------------- random draws ---------------- */

static uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xoshiro;

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xoshiro* x) {
  uint64_t* s = x->s;
  const uint64_t result = rotl(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

static void xo_seed(xoshiro* x, uint64_t seed) {
  uint64_t sm = seed;
  for (int i = 0; i < 4; ++i) x->s[i] = splitmix64(&sm);
}

/* uniform in [0, 1) from the top 53 bits */
static double xo_uniform(xoshiro* x) { return (double)(xo_next(x) >> 11) * (1.0 / 9007199254740992.0); }

/* first `count` outputs of SplitMix64 from state `seed` (tests of the generator) */
void cg_splitmix_raw(uint64_t seed, int64_t count, uint64_t* out) {
  uint64_t s = seed;
  for (int64_t i = 0; i < count; ++i) out[i] = splitmix64(&s);
}

/* xoshiro256** outputs from an explicit state (tests of the generator) */
void cg_xoshiro_from_state(const uint64_t* state, int64_t count, uint64_t* out) {
  xoshiro x;
  for (int i = 0; i < 4; ++i) x.s[i] = state[i];
  for (int64_t i = 0; i < count; ++i) out[i] = xo_next(&x);
}

/* raw stream access for tests of the generator itself */
void cg_rng_raw(uint64_t seed, int64_t count, uint64_t* out) {
  xoshiro x;
  xo_seed(&x, seed);
  for (int64_t i = 0; i < count; ++i) out[i] = xo_next(&x);
}

/* D_r = 10^U(lo_exp, hi_exp) for r < m, then b_k ~ N(0,1) for k < n (Box-Muller, both outputs used). */
void cg_draw_D_b(uint64_t seed, int64_t m, double lo_exp, double hi_exp, double* D, int64_t n, double* b) {
  xoshiro x;
  xo_seed(&x, seed);
  for (int64_t r = 0; r < m; ++r) {
    double u = xo_uniform(&x);
    D[r] = pow(10.0, lo_exp + (hi_exp - lo_exp) * u);
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t k = 0; k < n; k += 2) {
    double u1 = 1.0 - xo_uniform(&x); /* (0, 1] */
    double u2 = xo_uniform(&x);
    double rad = sqrt(-2.0 * log(u1));
    b[k] = rad * cos(two_pi * u2);
    if (k + 1 < n) b[k + 1] = rad * sin(two_pi * u2);
  }
}
