/*
 * Plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see ats_oracle.h).
 *
 * Written from the paper's equations: Eq. (Er_imp) / (Er_imp1) for the
 * backward-Euler finite-volume rows, the C coefficients of Sect. 3.1, the
 * Dirichlet / Neumann / Robin rows of Sect. 3.2, and the diagonal-
 * preconditioned CG with its L2 / L-infinity stopping rule of Sect. 3.3.4.
 * Every loop is the obvious one; nothing is blocked, fused or reordered.
 */
#include "ats_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- coordinate lookup by sorting (plain, obviously correct) ---------- */

typedef struct {
  int64_t key;
  int64_t idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b) {
  const keyidx *x = (const keyidx *)a, *y = (const keyidx *)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return 0;
}

/* pack non-negative-or-small-negative integer coordinates into one key */
static int64_t pack3(int64_t x, int64_t y, int64_t z) {
  const int64_t off = (int64_t)1 << 20; /* coordinates in (-2^20, 2^20) */
  return ((x + off) << 42) | ((y + off) << 21) | (z + off);
}

static int64_t lookup(const keyidx *tab, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (tab[mid].key == key) return tab[mid].idx;
    if (tab[mid].key < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

static const int DIR_AXIS[6] = {0, 0, 1, 1, 2, 2};
static const int DIR_SIGN[6] = {-1, +1, -1, +1, -1, +1};

int oracle_assemble(int64_t n_oct, const int32_t *oct_xyz, const uint8_t *leaf_mask, double dx,
                    double dt, const double *K, const double *s, const double *src,
                    const double *E_old, int64_t n_face, const int32_t *face_cell,
                    const int8_t *face_dir, const int8_t *face_kind, const int8_t *face_rel,
                    const double *face_alpha, const double *face_K, const double *face_E,
                    const double *face_F, int64_t *row_ptr, int32_t *col, double *val, double *b,
                    double *diag) {
  const int64_t N = 8 * n_oct;
  /* A^l = K dt / dx^2 with K the face mean (Sect. 3.1) */
  const double dt_dx2 = dt / (dx * dx);
  int rc = 0;

  keyidx *octs = (keyidx *)malloc(sizeof(keyidx) * (size_t)(n_oct > 0 ? n_oct : 1));
  keyidx *faces = (keyidx *)malloc(sizeof(keyidx) * (size_t)(n_face > 0 ? n_face : 1));
  if (!octs || !faces) {
    free(octs);
    free(faces);
    return -1;
  }
  for (int64_t o = 0; o < n_oct; ++o) {
    octs[o].key = pack3(oct_xyz[3 * o], oct_xyz[3 * o + 1], oct_xyz[3 * o + 2]);
    octs[o].idx = o;
  }
  qsort(octs, (size_t)n_oct, sizeof(keyidx), cmp_keyidx);
  for (int64_t o = 1; o < n_oct; ++o)
    if (octs[o].key == octs[o - 1].key) rc = -1; /* duplicate oct */

  for (int64_t f = 0; f < n_face; ++f) {
    if (face_cell[f] < 0 || face_cell[f] >= N || face_dir[f] < 0 || face_dir[f] > 5) rc = -1;
    faces[f].key = (int64_t)face_cell[f] * 6 + face_dir[f];
    faces[f].idx = f;
  }
  qsort(faces, (size_t)n_face, sizeof(keyidx), cmp_keyidx);
  for (int64_t f = 1; f < n_face; ++f)
    if (faces[f].key == faces[f - 1].key) rc = -1; /* duplicate descriptor */
  if (rc != 0) {
    free(octs);
    free(faces);
    return rc;
  }

  int64_t nnz = 0;
  for (int64_t i = 0; i < N; ++i) {
    const int64_t o = i / 8;
    const int c = (int)(i % 8);
    const int is_leaf = leaf_mask ? ((leaf_mask[o] >> c) & 1) : 1;
    row_ptr[i] = nnz;
    b[i] = 0.0;
    diag[i] = 0.0;
    if (!is_leaf) continue;
    if (!(K[i] > 0.0)) {
      rc = -1;
      continue;
    }

    /* level cell coordinates of cell i */
    const int64_t cx = 2 * (int64_t)oct_xyz[3 * o] + (c & 1);
    const int64_t cy = 2 * (int64_t)oct_xyz[3 * o + 1] + ((c >> 1) & 1);
    const int64_t cz = 2 * (int64_t)oct_xyz[3 * o + 2] + ((c >> 2) & 1);

    /* the "1" of Eq. (Er_imp1) plus the coupling shift */
    double d = 1.0 + (s ? s[i] : 0.0);
    double rhs = E_old[i] + (src ? src[i] : 0.0);
    const int64_t diag_pos = nnz; /* the diagonal entry goes first */
    col[nnz] = (int32_t)i;
    val[nnz] = 0.0;
    ++nnz;

    for (int dir = 0; dir < 6; ++dir) {
      int64_t nx = cx, ny = cy, nz = cz;
      if (DIR_AXIS[dir] == 0) nx += DIR_SIGN[dir];
      if (DIR_AXIS[dir] == 1) ny += DIR_SIGN[dir];
      if (DIR_AXIS[dir] == 2) nz += DIR_SIGN[dir];
      /* floor division by 2 for possibly negative coordinates */
      const int64_t nox = (nx >= 0) ? nx / 2 : -((-nx + 1) / 2);
      const int64_t noy = (ny >= 0) ? ny / 2 : -((-ny + 1) / 2);
      const int64_t noz = (nz >= 0) ? nz / 2 : -((-nz + 1) / 2);
      const int64_t no = lookup(octs, n_oct, pack3(nox, noy, noz));
      int64_t j = -1;
      if (no >= 0) {
        const int nc = (int)((nx - 2 * nox) + 2 * (ny - 2 * noy) + 4 * (nz - 2 * noz));
        const int nb_leaf = leaf_mask ? ((leaf_mask[no] >> nc) & 1) : 1;
        if (nb_leaf) j = 8 * no + nc;
      }
      const int64_t fid = lookup(faces, n_face, i * 6 + dir);
      if (j >= 0) {
        /* same-level leaf neighbour: C = A^l with K_{i+-1/2} = (K_i + K_j)/2 */
        if (fid >= 0) rc = -1; /* interior faces take no descriptor */
        const double C = dt_dx2 * 0.5 * (K[i] + K[j]);
        d += C;
        col[nnz] = (int32_t)j;
        val[nnz] = -C;
        ++nnz;
      } else if (fid >= 0) {
        /* interface face (Sect. 3.2): Dirichlet / Neumann / Robin */
        const double Kf = 0.5 * (K[i] + (face_K ? face_K[fid] : K[i]));
        const double factor = (face_rel[fid] == ORACLE_REL_COARSER) ? (2.0 / 3.0) : 1.0;
        const double C = factor * dt_dx2 * Kf;
        const double Enb = face_E ? face_E[fid] : 0.0;
        const double F = face_F ? face_F[fid] : 0.0;
        const double alpha = face_alpha ? face_alpha[fid] : 1.0;
        if (face_kind[fid] == ORACLE_DIRICHLET) {
          d += C;
          rhs += C * Enb;
        } else if (face_kind[fid] == ORACLE_NEUMANN) {
          rhs += F;
        } else if (face_kind[fid] == ORACLE_ROBIN) {
          if (alpha < 0.0 || alpha > 1.0) rc = -1;
          d += alpha * C;
          rhs += alpha * C * Enb + (1.0 - alpha) * F;
        } else {
          rc = -1;
        }
      }
      /* no neighbour and no descriptor: zero-flux wall, nothing added */
    }
    val[diag_pos] = d;
    diag[i] = d;
    b[i] = rhs;
  }
  row_ptr[N] = nnz;

  /* a descriptor on a non-leaf cell is an error too */
  for (int64_t f = 0; f < n_face; ++f) {
    const int64_t i = face_cell[f];
    const int64_t o = i / 8;
    const int c = (int)(i % 8);
    if (leaf_mask && !((leaf_mask[o] >> c) & 1)) rc = -1;
  }
  free(octs);
  free(faces);
  return rc;
}

/* ---- compensated sums ------------------------------------------------- */

typedef struct {
  double s, c;
} nsum;

static void nsum_add(nsum *a, double v) {
  /* Neumaier's improved Kahan-Babuska summation */
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

void oracle_matvec(int64_t N, const int64_t *row_ptr, const int32_t *col, const double *val,
                   const double *x, double *y) {
  for (int64_t i = 0; i < N; ++i) {
    double acc = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) acc += val[k] * x[col[k]];
    y[i] = acc;
  }
}

double oracle_residual(int64_t N, const int64_t *row_ptr, const int32_t *col, const double *val,
                       const double *b, const double *x, double *r) {
  nsum norm = {0.0, 0.0};
  for (int64_t i = 0; i < N; ++i) {
    if (row_ptr[i + 1] == row_ptr[i]) {
      r[i] = 0.0;
      continue;
    }
    nsum acc = {0.0, 0.0};
    nsum_add(&acc, b[i]);
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) nsum_add(&acc, -val[k] * x[col[k]]);
    r[i] = nsum_get(&acc);
    nsum_add(&norm, r[i] * r[i]);
  }
  return sqrt(nsum_get(&norm));
}

static double dot_rows(int64_t N, const int64_t *row_ptr, const double *a, const double *b) {
  double acc = 0.0;
  for (int64_t i = 0; i < N; ++i)
    if (row_ptr[i + 1] > row_ptr[i]) acc += a[i] * b[i];
  return acc;
}

/* Jacobi-preconditioned CG, Sect. 3.3.4: diagonal preconditioner, stop on
 * ||r_j||/||r_0|| < eps and (paper rule) max |E_j - E_{j-1}| / E_{j-1} < eps. */
int oracle_pcg(int64_t N, const int64_t *row_ptr, const int32_t *col, const double *val,
               const double *diag, const double *b, double *x, double tol, int stop_rule,
               int64_t max_iter, double *info) {
  double *r = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
  double *z = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
  double *p = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
  double *q = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
  int rc = 1;
  int64_t it = 0;
  double maxchg = 0.0;
  if (!r || !z || !p || !q) {
    free(r);
    free(z);
    free(p);
    free(q);
    return -1;
  }

  const double r0 = oracle_residual(N, row_ptr, col, val, b, x, r);
  double rnorm = r0;
  info[1] = r0;
  if (r0 == 0.0) {
    rc = 0;
  } else {
    for (int64_t i = 0; i < N; ++i) {
      const int leaf = row_ptr[i + 1] > row_ptr[i];
      z[i] = leaf ? r[i] / diag[i] : 0.0;
      p[i] = z[i];
    }
    double rz = dot_rows(N, row_ptr, r, z);
    while (it < max_iter) {
      oracle_matvec(N, row_ptr, col, val, p, q);
      const double pq = dot_rows(N, row_ptr, p, q);
      if (!(pq > 0.0)) {
        rc = -1;
        break;
      }
      const double alpha = rz / pq;
      maxchg = 0.0;
      for (int64_t i = 0; i < N; ++i) {
        if (row_ptr[i + 1] == row_ptr[i]) continue;
        const double step = alpha * p[i];
        const double chg = fabs(step) / fabs(x[i]);
        if (chg > maxchg || chg != chg) maxchg = chg;
        x[i] += step;
        r[i] -= alpha * q[i];
      }
      ++it;
      rnorm = sqrt(dot_rows(N, row_ptr, r, r));
      int done;
      if (stop_rule == ORACLE_STOP_CERTIFIED) {
        const double xnorm = sqrt(dot_rows(N, row_ptr, x, x));
        done = rnorm <= tol * xnorm;
        if (done) {
          /* confirm with the true residual; if rounding hid it, restart CG
           * from the true residual (p = z) and go on */
          const double tr = oracle_residual(N, row_ptr, col, val, b, x, r);
          done = tr <= tol * xnorm;
          if (!done) {
            for (int64_t i = 0; i < N; ++i) {
              z[i] = (row_ptr[i + 1] > row_ptr[i]) ? r[i] / diag[i] : 0.0;
              p[i] = z[i];
            }
            rz = dot_rows(N, row_ptr, r, z);
            continue;
          }
        }
      } else if (stop_rule == ORACLE_STOP_PAPER) {
        done = (rnorm / r0 < tol) && (maxchg < tol);
      } else {
        done = rnorm / r0 < tol;
      }
      if (done) {
        rc = 0;
        break;
      }
      for (int64_t i = 0; i < N; ++i)
        z[i] = (row_ptr[i + 1] > row_ptr[i]) ? r[i] / diag[i] : 0.0;
      const double rz_new = dot_rows(N, row_ptr, r, z);
      if (!(rz_new > 0.0) || rz_new != rz_new) {
        rc = -1;
        break;
      }
      const double beta = rz_new / rz;
      rz = rz_new;
      for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
  }
  info[0] = (double)it;
  info[2] = oracle_residual(N, row_ptr, col, val, b, x, r);
  info[3] = sqrt(dot_rows(N, row_ptr, x, x));
  info[4] = maxchg;
  free(r);
  free(z);
  free(p);
  free(q);
  return rc;
}
