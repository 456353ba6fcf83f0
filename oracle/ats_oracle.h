/*
 * Plain FP64 CPU oracle for the per-level implicit diffusion solve of
 * Commerçon, Debout & Teyssier (2014), "A fast, robust, and simple implicit
 * method for adaptive time-stepping on AMR grids".
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load or call this code.  The
 * product path (the CUDA library) shares no code, header, table or helper with
 * it, and neither side includes or links the other.
 *
 * What it computes (all FP64, no blocking, fusion or reordering):
 *   - oracle_assemble: the level matrix of Eq. (Er_imp1) in 3D, one row per
 *     leaf cell, with the face coefficients C of Sect. 3.1 (C^{l->l} and
 *     C^{l->l+1} = A^l, C^{l->l-1} = 2/3 A^l) and the interface rows of
 *     Sect. 3.2 (Dirichlet, Neumann, Robin), written out as explicit CSR.
 *   - oracle_pcg: conjugate gradient with a diagonal (Jacobi) preconditioner
 *     and the stopping rules of Sect. 3.3.4 ("Implicit update").
 *   - oracle_residual: r = b - A x with compensated (Neumaier) summation.
 *
 * Cell numbering: a level is a list of octs (2x2x2 cells).  Oct o has integer
 * oct coordinates (ox, oy, oz); its cell c = ix + 2 iy + 4 iz (ix, iy, iz in
 * {0,1}) has level cell coordinates (2 ox + ix, 2 oy + iy, 2 oz + iz) and the
 * global index 8 o + c.  Face directions: 0 = -x, 1 = +x, 2 = -y, 3 = +y,
 * 4 = -z, 5 = +z.
 */
#ifndef ATS_ORACLE_H
#define ATS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* face kinds (Sect. 3.2) */
#define ORACLE_DIRICHLET 0
#define ORACLE_NEUMANN 1
#define ORACLE_ROBIN 2
/* face relations (Sect. 3.1): distance factor 1 or 2/3 */
#define ORACLE_REL_SAME 0    /* physical ghost at distance dx, factor 1 */
#define ORACLE_REL_COARSER 1 /* fine-to-coarse, factor 2/3 */
#define ORACLE_REL_FINER 2   /* coarse-to-fine (restricted finer cell), factor 1 */

/* stopping rules (Sect. 3.3.4) */
#define ORACLE_STOP_RESIDUAL 0  /* ||r_j|| / ||r_0|| < tol */
#define ORACLE_STOP_CERTIFIED 1 /* ||b - A x|| <= tol ||x||  (relative error <= tol, lambda_min >= 1) */
#define ORACLE_STOP_PAPER 2     /* L2 rule AND max |x_j - x_{j-1}| / |x_{j-1}| < tol */

/*
 * Assemble the level system.  Arrays are host arrays; N = 8 n_oct.
 *   K[N]            cell diffusion coefficient (> 0 on leaf cells)
 *   s[N] or NULL    extra diagonal (linearised coupling shift), 0 if NULL
 *   src[N] or NULL  extra right-hand side, 0 if NULL
 *   E_old[N]        E^n, the right-hand side base
 *   face_*          interface descriptors for faces that have no same-level
 *                   leaf neighbour; a face with no descriptor is a zero-flux
 *                   wall (nothing added).  face_K / face_E / face_F / face_alpha
 *                   may be NULL (K of the cell / 0 / 0 / 1).
 * Outputs: row_ptr[N+1], col[7N], val[7N], b[N], diag[N].  Non-leaf cells get
 * an empty row, b = 0 and diag = 0.
 * Returns 0, or -1 on an invalid description (descriptor on an interior face,
 * duplicate descriptor, bad index, non-positive K on a leaf).
 */
int oracle_assemble(int64_t n_oct, const int32_t *oct_xyz, const uint8_t *leaf_mask, double dx,
                    double dt, const double *K, const double *s, const double *src,
                    const double *E_old, int64_t n_face, const int32_t *face_cell,
                    const int8_t *face_dir, const int8_t *face_kind, const int8_t *face_rel,
                    const double *face_alpha, const double *face_K, const double *face_E,
                    const double *face_F, int64_t *row_ptr, int32_t *col, double *val, double *b,
                    double *diag);

/* r = b - A x over leaf rows (non-leaf rows: r = 0); returns ||r||_2.
 * Row sums and the norm use Neumaier compensated summation. */
double oracle_residual(int64_t N, const int64_t *row_ptr, const int32_t *col, const double *val,
                       const double *b, const double *x, double *r);

/* Jacobi-preconditioned CG on the leaf rows; x holds x_0 on entry and the
 * solution on exit (non-leaf entries are left as they are).
 * info[0] = iterations, info[1] = ||r_0||, info[2] = final ||b - A x|| (true),
 * info[3] = ||x||, info[4] = last max relative change.  Returns 0 on
 * convergence, 1 if max_iter was reached, -1 on breakdown (p.Ap <= 0). */
int oracle_pcg(int64_t N, const int64_t *row_ptr, const int32_t *col, const double *val,
               const double *diag, const double *b, double *x, double tol, int stop_rule,
               int64_t max_iter, double *info);

/* y = A x (leaf rows only; non-leaf rows give 0). */
void oracle_matvec(int64_t N, const int64_t *row_ptr, const int32_t *col, const double *val,
                   const double *x, double *y);

#ifdef __cplusplus
}
#endif
#endif
