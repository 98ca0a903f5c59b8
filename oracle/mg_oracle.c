/*
 * mg_oracle.c -- plain, slow FP64 CPU oracle of the masked-domain multigrid
 * Poisson solver of Guillet & Teyssier, "A Simple Multigrid Scheme for Solving
 * the Poisson Equation with Arbitrary Domain Boundaries" (arXiv:1104.1703).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this library.  The product path (the CUDA
 * library under paper_1104_1703_gb300/csrc) shares no code with it and never
 * calls it.
 *
 * The code follows the paper's steps in its order and notation, with straight
 * loops and no folding: ghost values are built literally (Section 3, Fig. 5),
 * the residual is r = Laplacian(Phi) - rho (Section 2, recipe step 2), the
 * coarse problem is Laplacian_c(dPhi_c) = -R(r) with dPhi_c = 0 on the coarse
 * boundary (recipe step 5), R is R1 and P is P2 (Fig. 3).
 *
 * Storage: cell-centred grids, x fastest, idx = (k*ny + j)*nx + i.  The mask of
 * level l is kept as the integer sum S_l of the level-0 colours (+1 inside, -1
 * outside) so that m_l = S_l / 8^l is exact (Section 3, mask averaging).
 *
 * Readings where the paper is silent (each listed in the design notes):
 *  - red = (i+j+k) even is swept first, in every sweep;
 *  - out-of-box cells have m = -1 at every level, and missing children of an
 *    odd-sized level count as m = -1 (mask) and r = 0 (residual);
 *  - first-order mode applies on levels l >= 1 only; level 0 keeps its
 *    Dirichlet faces;
 *  - P2 reads the stored value 0 at coarse cells outside Omega_c and at
 *    out-of-box coarse indices;
 *  - the deepest level with an active cell gets a fixed number of red-black
 *    sweeps (coarse_sweeps) instead of a further coarse grid;
 *  - order switch: see orc_solve.
 *
 * Parity status: every function below is pinned by the CPU tests (closed
 * forms, worked figure values, dense direct solve, convergence order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXL 16

/* ------------------------------------------------------------------------ */
/* Small helpers                                                             */
/* ------------------------------------------------------------------------ */

static int64_t pow8(int l) {
  int64_t p = 1;
  while (l-- > 0) p *= 8;
  return p;
}

static size_t cell(int i, int j, int k, int nx, int ny) {
  return ((size_t)k * ny + j) * nx + i;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Section 3: Omega^l = {m^l > 0}.  Section 4: in first-order mode the
 * constraint Phi = 0 is imposed on every coarse cell with m < 1, so the
 * unknowns are the cells with m = 1 exactly, i.e. S = 8^l. */
int orc_is_active(int64_t S, int level, int order) {
  if (level >= 1 && order == 1) return S == pow8(level);
  return S > 0;
}

/* Section 3 / Fig. 5: the boundary sits where the linearly interpolated mask
 * crosses zero between the centre of cell i (m_i > 0) and of neighbour j
 * (m_j <= 0).  theta is the distance from i to that point in units of the
 * cell size. */
double orc_theta(double m_i, double m_j) { return m_i / (m_i - m_j); }

/* Section 3 / Fig. 5: ghost value linearly extrapolated from Phi_i through
 * the boundary value Phi_b located at distance theta. */
double orc_ghost(double phi_i, double phi_b, double theta) {
  return phi_i + (phi_b - phi_i) / theta;
}

/* ------------------------------------------------------------------------ */
/* Neighbour classification for the modified Laplacian (Sections 3 and 4)    */
/* ------------------------------------------------------------------------ */

enum { NB_ACTIVE = 0, NB_GHOST = 1, NB_NGP_ZERO = 2 };

typedef struct {
  int kind;      /* NB_ACTIVE, NB_GHOST or NB_NGP_ZERO */
  double phi_j;  /* neighbour value (NB_ACTIVE) */
  double theta;  /* boundary distance (NB_GHOST) */
  double phi_b;  /* boundary value (NB_GHOST) */
} nb_info;

/* Direction d: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z.
 * bx, by, bz are the level-0 face values (NULL means zero); they are only
 * read at level 0.  At coarse levels the correction problem has Phi_b = 0
 * (recipe step 5). */
static nb_info classify(int nx, int ny, int nz, int level, const int64_t* S, int order,
                        const double* phi, const double* bx, const double* by,
                        const double* bz, int i, int j, int k, int d) {
  static const int dx[6] = {-1, 1, 0, 0, 0, 0};
  static const int dy[6] = {0, 0, -1, 1, 0, 0};
  static const int dz[6] = {0, 0, 0, 0, -1, 1};
  const int64_t p8 = pow8(level);
  int ii = i + dx[d], jj = j + dy[d], kk = k + dz[d];
  int inside = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
  int64_t Sj = inside ? S[cell(ii, jj, kk, nx, ny)] : -p8;
  nb_info nb;
  nb.phi_j = 0.0;
  nb.theta = 1.0;
  nb.phi_b = 0.0;
  if (orc_is_active(Sj, level, order)) {
    nb.kind = NB_ACTIVE;
    nb.phi_j = phi[cell(ii, jj, kk, nx, ny)];
    return nb;
  }
  if (level >= 1 && order == 1) {
    /* Section 4 (NGP): the neighbour carries the constraint Phi = 0 at its
     * own centre. */
    nb.kind = NB_NGP_ZERO;
    return nb;
  }
  nb.kind = NB_GHOST;
  {
    double m_i = (double)S[cell(i, j, k, nx, ny)] / (double)p8;
    double m_j = (double)Sj / (double)p8;
    nb.theta = orc_theta(m_i, m_j);
  }
  if (level == 0) {
    /* Fig. 1: boundary values live on the border faces of the fine level. */
    double v = 0.0;
    if (d == 0 && bx) v = bx[((size_t)k * ny + j) * (nx + 1) + i];
    if (d == 1 && bx) v = bx[((size_t)k * ny + j) * (nx + 1) + i + 1];
    if (d == 2 && by) v = by[((size_t)k * (ny + 1) + j) * nx + i];
    if (d == 3 && by) v = by[((size_t)k * (ny + 1) + j + 1) * nx + i];
    if (d == 4 && bz) v = bz[((size_t)k * ny + j) * nx + i];
    if (d == 5 && bz) v = bz[((size_t)(k + 1) * ny + j) * nx + i];
    nb.phi_b = v;
  }
  return nb;
}

/* ------------------------------------------------------------------------ */
/* Operators                                                                 */
/* ------------------------------------------------------------------------ */

/* Section 2, 7-point Laplacian, with the modified stencil of Section 3 (ghost
 * values across the boundary) or, in first-order mode on coarse levels, the
 * NGP constraint of Section 4.  out = (Laplacian Phi) on active cells, 0
 * elsewhere.  hl is the cell size of this level. */
void orc_laplacian(int nx, int ny, int nz, int level, const int64_t* S, int order, double hl,
                   const double* phi, const double* bx, const double* by, const double* bz,
                   double* out) {
  const double h2 = hl * hl;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = cell(i, j, k, nx, ny);
        if (!orc_is_active(S[c], level, order)) {
          out[c] = 0.0;
          continue;
        }
        double phi_i = phi[c];
        double lap = 0.0;
        for (int d = 0; d < 6; ++d) {
          nb_info nb = classify(nx, ny, nz, level, S, order, phi, bx, by, bz, i, j, k, d);
          double phi_star;
          if (nb.kind == NB_ACTIVE)
            phi_star = nb.phi_j;
          else if (nb.kind == NB_GHOST)
            phi_star = orc_ghost(phi_i, nb.phi_b, nb.theta);
          else
            phi_star = 0.0;
          lap += (phi_star - phi_i) / h2;
        }
        out[c] = lap;
      }
}

/* Section 2, recipe step 2: r = Laplacian(Phi) - rho on active cells, 0
 * elsewhere. */
void orc_residual(int nx, int ny, int nz, int level, const int64_t* S, int order, double hl,
                  const double* phi, const double* rho, const double* bx, const double* by,
                  const double* bz, double* r) {
  orc_laplacian(nx, ny, nz, level, S, order, hl, phi, bx, by, bz, r);
  size_t n = (size_t)nx * ny * nz;
  for (size_t c = 0; c < n; ++c)
    if (orc_is_active(S[c], level, order)) r[c] -= rho[c];
}

/* One Gauss-Seidel update of cell (i,j,k): the cell's own equation
 * (Laplacian Phi)_i = rho_i is solved for Phi_i with the neighbours held
 * fixed.  Each neighbour direction contributes (a - c*Phi_i)/h^2 with
 *   active neighbour:  a = Phi_j,          c = 1
 *   ghost (Fig. 5):    a = Phi_b / theta,  c = 1 / theta
 *   NGP zero (Sec. 4): a = 0,              c = 1
 * which is the literal ghost term (ghost(Phi_i) - Phi_i)/h^2 rewritten. */
static void gs_update(int nx, int ny, int nz, int level, const int64_t* S, int order, double h2,
                      double* phi, const double* rho, const double* bx, const double* by,
                      const double* bz, int i, int j, int k) {
  size_t c = cell(i, j, k, nx, ny);
  double sum_a = 0.0, sum_c = 0.0;
  for (int d = 0; d < 6; ++d) {
    nb_info nb = classify(nx, ny, nz, level, S, order, phi, bx, by, bz, i, j, k, d);
    if (nb.kind == NB_ACTIVE) {
      sum_a += nb.phi_j;
      sum_c += 1.0;
    } else if (nb.kind == NB_GHOST) {
      sum_a += nb.phi_b / nb.theta;
      sum_c += 1.0 / nb.theta;
    } else {
      sum_c += 1.0;
    }
  }
  phi[c] = (sum_a - h2 * rho[c]) / sum_c;
}

/* Section 2: Gauss-Seidel smoother with red-black ordering; one sweep is a
 * pass over the red cells ((i+j+k) even) followed by a pass over the black
 * cells.  Only active cells are updated. */
void orc_gs_sweeps(int nx, int ny, int nz, int level, const int64_t* S, int order, double hl,
                   double* phi, const double* rho, const double* bx, const double* by,
                   const double* bz, int sweeps) {
  const double h2 = hl * hl;
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for schedule(static)
      for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
          for (int i = 0; i < nx; ++i) {
            if (((i + j + k) & 1) != colour) continue;
            if (!orc_is_active(S[cell(i, j, k, nx, ny)], level, order)) continue;
            gs_update(nx, ny, nz, level, S, order, h2, phi, rho, bx, by, bz, i, j, k);
          }
    }
}

/* Section 3: the mask of the next coarser level is the R1 average of its
 * children, applied recursively; in integer form Sc = sum of the 8 children.
 * Coarse dimensions are ceil(n/2); a missing child (odd dimension) lies
 * outside the box and counts as m = -1.  Returns the number of cells with
 * Sc > 0. */
long orc_mask_restrict(int nx, int ny, int nz, int level, const int64_t* S, int64_t* Sc) {
  int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
  const int64_t p8 = pow8(level);
  long n_pos = 0;
  for (int K = 0; K < cz; ++K)
    for (int J = 0; J < cy; ++J)
      for (int I = 0; I < cx; ++I) {
        int64_t sum = 0;
        for (int c = 0; c < 8; ++c) {
          int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + ((c >> 2) & 1);
          int inside = i < nx && j < ny && k < nz;
          sum += inside ? S[cell(i, j, k, nx, ny)] : -p8;
        }
        Sc[cell(I, J, K, cx, cy)] = sum;
        if (sum > 0) ++n_pos;
      }
  return n_pos;
}

/* Fig. 3, R1: the coarse value is the average of the 8 children (1/4 each in
 * the 2D figure, 1/8 in 3D).  Missing children of an odd dimension carry 0. */
void orc_restrict(int nx, int ny, int nz, const double* r, double* rc) {
  int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
#pragma omp parallel for schedule(static)
  for (int K = 0; K < cz; ++K)
    for (int J = 0; J < cy; ++J)
      for (int I = 0; I < cx; ++I) {
        double sum = 0.0;
        for (int c = 0; c < 8; ++c) {
          int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + ((c >> 2) & 1);
          if (i < nx && j < ny && k < nz) sum += r[cell(i, j, k, nx, ny)];
        }
        rc[cell(I, J, K, cx, cy)] = sum / 8.0;
      }
}

/* One axis of P2 (Fig. 3): a fine cell centre lies a quarter of a coarse cell
 * from its parent's centre, so it takes 3/4 of the parent and 1/4 of the
 * coarse neighbour on its side. */
static void p2_axis(int i, int* lo, double* w_lo, double* w_hi) {
  int I = i >> 1;
  if ((i & 1) == 0) {
    *lo = I - 1;
    *w_lo = 0.25;
    *w_hi = 0.75;
  } else {
    *lo = I;
    *w_lo = 0.75;
    *w_hi = 0.25;
  }
}

/* Fig. 3, P2 (bilinear in the figure, trilinear here) and recipe steps 6-7:
 * Phi_f += P(dPhi_c) on the active fine cells.  The coarse values outside
 * the coarse box count as 0. */
void orc_prolong_add(int cx, int cy, int cz, const double* ec, int nx, int ny, int nz, int level_f,
                     const int64_t* Sf, int order, double* phi) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = cell(i, j, k, nx, ny);
        if (!orc_is_active(Sf[c], level_f, order)) continue;
        int xi, yj, zk;
        double wx[2], wy[2], wz[2];
        p2_axis(i, &xi, &wx[0], &wx[1]);
        p2_axis(j, &yj, &wy[0], &wy[1]);
        p2_axis(k, &zk, &wz[0], &wz[1]);
        double corr = 0.0;
        for (int c3 = 0; c3 < 8; ++c3) {
          int a = c3 & 1, b = (c3 >> 1) & 1, e = (c3 >> 2) & 1;
          int I = xi + a, J = yj + b, K = zk + e;
          if (I < 0 || I >= cx || J < 0 || J >= cy || K < 0 || K >= cz) continue;
          corr += wx[a] * wy[b] * wz[e] * ec[cell(I, J, K, cx, cy)];
        }
        phi[c] += corr;
      }
}

/* Fig. 1 caption and Section 1 (one-way interface): the Dirichlet values on
 * the border faces of the fine level are linearly interpolated from the
 * solution of the coarser AMR level.  The coarse grid has cell size 2h; its
 * cell (I,J,K) spans [o + 2I, o + 2I + 2] in fine-cell units, so its centre is
 * at o + 2I + 1.  The value at a face centre is the trilinear interpolation
 * of the 8 surrounding coarse centres.  Only faces between an active cell
 * and an inactive or out-of-box cell are filled; the others are set to 0.
 * Returns 0, or -1 if a needed face falls outside the coarse centres. */
static int trilinear_at(const double* pc, int cnx, int cny, int cnz, int ox, int oy, int oz,
                        double px, double py, double pz, double* out) {
  double u = (px - ox) / 2.0 - 0.5, v = (py - oy) / 2.0 - 0.5, w = (pz - oz) / 2.0 - 0.5;
  int I = (int)floor(u), J = (int)floor(v), K = (int)floor(w);
  double tu = u - I, tv = v - J, tw = w - K;
  if (I < 0 || J < 0 || K < 0 || I + 1 >= cnx || J + 1 >= cny || K + 1 >= cnz) return -1;
  double val = 0.0;
  for (int c = 0; c < 8; ++c) {
    int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
    double wgt = (a ? tu : 1.0 - tu) * (b ? tv : 1.0 - tv) * (e ? tw : 1.0 - tw);
    val += wgt * pc[cell(I + a, J + b, K + e, cnx, cny)];
  }
  *out = val;
  return 0;
}

int orc_dirichlet_from_coarse(int nx, int ny, int nz, const int8_t* mask, const double* pc,
                              int cnx, int cny, int cnz, int ox, int oy, int oz, double* bx,
                              double* by, double* bz) {
  int status = 0;
  memset(bx, 0, sizeof(double) * (size_t)(nx + 1) * ny * nz);
  memset(by, 0, sizeof(double) * (size_t)nx * (ny + 1) * nz);
  memset(bz, 0, sizeof(double) * (size_t)nx * ny * (nz + 1));
#define ACT(i, j, k) \
  ((i) >= 0 && (i) < nx && (j) >= 0 && (j) < ny && (k) >= 0 && (k) < nz && mask[cell(i, j, k, nx, ny)] > 0)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i)
        if (ACT(i - 1, j, k) != ACT(i, j, k))
          if (trilinear_at(pc, cnx, cny, cnz, ox, oy, oz, i, j + 0.5, k + 0.5,
                           &bx[((size_t)k * ny + j) * (nx + 1) + i]))
            status = -1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i)
        if (ACT(i, j - 1, k) != ACT(i, j, k))
          if (trilinear_at(pc, cnx, cny, cnz, ox, oy, oz, i + 0.5, j, k + 0.5,
                           &by[((size_t)k * (ny + 1) + j) * nx + i]))
            status = -1;
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        if (ACT(i, j, k - 1) != ACT(i, j, k))
          if (trilinear_at(pc, cnx, cny, cnz, ox, oy, oz, i + 0.5, j + 0.5, k,
                           &bz[((size_t)k * ny + j) * nx + i]))
            status = -1;
#undef ACT
  return status;
}

/* L2 norm over the active cells, summed in index order. */
static double norm2_active(size_t n, const int64_t* S, int level, int order, const double* r) {
  double s = 0.0;
  for (size_t c = 0; c < n; ++c)
    if (orc_is_active(S[c], level, order)) s += r[c] * r[c];
  return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Hierarchy, V-cycle and solve                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nlev;
  int nx[ORC_MAXL], ny[ORC_MAXL], nz[ORC_MAXL];
  int64_t* S[ORC_MAXL];
  double* phi[ORC_MAXL]; /* level 0: Phi; level >= 1: the correction dPhi */
  double* rhs[ORC_MAXL]; /* level 0: rho; level >= 1: -R(r) */
  double* res[ORC_MAXL];
  long n_active[3][ORC_MAXL]; /* [order][level] */
  int deepest[3];             /* deepest level with an active cell, per order */
  double h;
  double *bx, *by, *bz;
  int hold; /* solves left in forced first-order mode (Section 4) */
} orc_hier;

static size_t ncells(const orc_hier* H, int l) { return (size_t)H->nx[l] * H->ny[l] * H->nz[l]; }

void orc_destroy(orc_hier* H) {
  if (!H) return;
  for (int l = 0; l < H->nlev; ++l) {
    free(H->S[l]);
    free(H->phi[l]);
    free(H->rhs[l]);
    free(H->res[l]);
  }
  free(H->bx);
  free(H->by);
  free(H->bz);
  free(H);
}

/* Section 2 (Fig. 2) and Section 3: the hierarchy of coarse grids covering the
 * fine domain.  Levels are built by halving (ceil) until every dimension is at
 * most 2.  The mask of level 0 is +1 on active cells (mask > 0) and -1
 * elsewhere. */
orc_hier* orc_create(const int8_t* mask, int nx, int ny, int nz, double h) {
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0)) return NULL;
  orc_hier* H = (orc_hier*)calloc(1, sizeof(orc_hier));
  H->h = h;
  H->nx[0] = nx;
  H->ny[0] = ny;
  H->nz[0] = nz;
  int l = 0;
  for (;;) {
    size_t n = (size_t)H->nx[l] * H->ny[l] * H->nz[l];
    H->S[l] = (int64_t*)calloc(n, sizeof(int64_t));
    H->phi[l] = (double*)calloc(n, sizeof(double));
    H->rhs[l] = (double*)calloc(n, sizeof(double));
    H->res[l] = (double*)calloc(n, sizeof(double));
    H->nlev = l + 1;
    if ((H->nx[l] <= 2 && H->ny[l] <= 2 && H->nz[l] <= 2) || l + 1 >= ORC_MAXL) break;
    H->nx[l + 1] = (H->nx[l] + 1) / 2;
    H->ny[l + 1] = (H->ny[l] + 1) / 2;
    H->nz[l + 1] = (H->nz[l] + 1) / 2;
    ++l;
  }
  size_t n0 = (size_t)nx * ny * nz;
  for (size_t c = 0; c < n0; ++c) H->S[0][c] = mask[c] > 0 ? 1 : -1;
  for (l = 0; l + 1 < H->nlev; ++l)
    orc_mask_restrict(H->nx[l], H->ny[l], H->nz[l], l, H->S[l], H->S[l + 1]);
  for (int order = 1; order <= 2; ++order) {
    H->deepest[order] = -1;
    for (l = 0; l < H->nlev; ++l) {
      long cnt = 0;
      for (size_t c = 0; c < ncells(H, l); ++c) cnt += orc_is_active(H->S[l][c], l, order);
      H->n_active[order][l] = cnt;
    }
    for (l = 0; l < H->nlev && H->n_active[order][l] > 0; ++l) H->deepest[order] = l;
  }
  if (H->deepest[2] < 0) {
    orc_destroy(H);
    return NULL;
  }
  H->bx = (double*)calloc((size_t)(nx + 1) * ny * nz, sizeof(double));
  H->by = (double*)calloc((size_t)nx * (ny + 1) * nz, sizeof(double));
  H->bz = (double*)calloc((size_t)nx * ny * (nz + 1), sizeof(double));
  return H;
}

int orc_num_levels(const orc_hier* H) { return H->nlev; }
int orc_deepest(const orc_hier* H, int order) { return H->deepest[order]; }
long orc_level_active(const orc_hier* H, int level, int order) { return H->n_active[order][level]; }
void orc_level_dims(const orc_hier* H, int level, int* d) {
  d[0] = H->nx[level];
  d[1] = H->ny[level];
  d[2] = H->nz[level];
}
int orc_get_hold(const orc_hier* H) { return H->hold; }
void orc_set_hold(orc_hier* H, int hold) { H->hold = hold; }

/* field: 0 S (int64), 1 phi, 2 rhs, 3 res */
void* orc_level_ptr(orc_hier* H, int level, int field) {
  switch (field) {
    case 0: return H->S[level];
    case 1: return H->phi[level];
    case 2: return H->rhs[level];
    case 3: return H->res[level];
  }
  return NULL;
}

static double level_h(const orc_hier* H, int l) { return ldexp(H->h, l); }

void orc_set_rhs(orc_hier* H, const double* rho) {
  size_t n = ncells(H, 0);
  for (size_t c = 0; c < n; ++c) H->rhs[0][c] = H->S[0][c] > 0 ? rho[c] : 0.0;
}

void orc_set_faces(orc_hier* H, const double* bx, const double* by, const double* bz) {
  int nx = H->nx[0], ny = H->ny[0], nz = H->nz[0];
  size_t fx = (size_t)(nx + 1) * ny * nz, fy = (size_t)nx * (ny + 1) * nz, fz = (size_t)nx * ny * (nz + 1);
  if (bx) memcpy(H->bx, bx, fx * sizeof(double)); else memset(H->bx, 0, fx * sizeof(double));
  if (by) memcpy(H->by, by, fy * sizeof(double)); else memset(H->by, 0, fy * sizeof(double));
  if (bz) memcpy(H->bz, bz, fz * sizeof(double)); else memset(H->bz, 0, fz * sizeof(double));
}

void orc_set_phi(orc_hier* H, const double* phi) {
  size_t n = ncells(H, 0);
  for (size_t c = 0; c < n; ++c) H->phi[0][c] = (phi && H->S[0][c] > 0) ? phi[c] : 0.0;
}

void orc_get_phi(const orc_hier* H, double* phi) { memcpy(phi, H->phi[0], ncells(H, 0) * sizeof(double)); }

/* Level operators on the hierarchy's own arrays (used by the recursion and
 * exposed for per-operator comparisons). */
void orc_level_smooth(orc_hier* H, int l, int order, int sweeps) {
  orc_gs_sweeps(H->nx[l], H->ny[l], H->nz[l], l, H->S[l], order, level_h(H, l), H->phi[l], H->rhs[l],
                l == 0 ? H->bx : NULL, l == 0 ? H->by : NULL, l == 0 ? H->bz : NULL, sweeps);
}

double orc_level_residual(orc_hier* H, int l, int order) {
  orc_residual(H->nx[l], H->ny[l], H->nz[l], l, H->S[l], order, level_h(H, l), H->phi[l], H->rhs[l],
               l == 0 ? H->bx : NULL, l == 0 ? H->by : NULL, l == 0 ? H->bz : NULL, H->res[l]);
  return norm2_active(ncells(H, l), H->S[l], l, order, H->res[l]);
}

/* Recipe steps 2-3 and 5: residual of level l, then rhs_{l+1} = -R1(r) and
 * dPhi_{l+1} = 0 as the start of the coarse correction problem. */
void orc_level_restrict(orc_hier* H, int l, int order) {
  orc_level_residual(H, l, order);
  orc_restrict(H->nx[l], H->ny[l], H->nz[l], H->res[l], H->rhs[l + 1]);
  size_t n = ncells(H, l + 1);
  for (size_t c = 0; c < n; ++c) {
    H->rhs[l + 1][c] = -H->rhs[l + 1][c];
    H->phi[l + 1][c] = 0.0;
  }
}

/* Recipe steps 6-7. */
void orc_level_prolong(orc_hier* H, int l, int order) {
  orc_prolong_add(H->nx[l + 1], H->ny[l + 1], H->nz[l + 1], H->phi[l + 1], H->nx[l], H->ny[l],
                  H->nz[l], l, H->S[l], order, H->phi[l]);
}

/* Section 2 recipe, applied recursively (N_cycles coarse iterations per
 * level, Section 5.3).  The deepest level with an active cell is smoothed
 * coarse_sweeps times instead of being coarsened further. */
static void mg_iteration(orc_hier* H, int l, int order, int n_pre, int n_post, int n_cycles,
                         int coarse_sweeps) {
  if (l == H->deepest[order]) {
    orc_level_smooth(H, l, order, coarse_sweeps);
    return;
  }
  orc_level_smooth(H, l, order, n_pre);                 /* step 1 */
  orc_level_restrict(H, l, order);                      /* steps 2-4 */
  for (int c = 0; c < n_cycles; ++c)                    /* step 5 */
    mg_iteration(H, l + 1, order, n_pre, n_post, n_cycles, coarse_sweeps);
  orc_level_prolong(H, l, order);                       /* steps 6-7 */
  orc_level_smooth(H, l, order, n_post);                /* step 8 */
}

void orc_vcycle(orc_hier* H, int order, int n_pre, int n_post, int n_cycles, int coarse_sweeps) {
  mg_iteration(H, 0, order, n_pre, n_post, n_cycles, coarse_sweeps);
}

/* L2 norm of the fine residual r = Laplacian(Phi) - rho over active cells. */
double orc_residual_norm(orc_hier* H) { return orc_level_residual(H, 0, 2); }

/* Norm of the residual of the zero field, the reference of the relative
 * residual (Section 5.2 measures the residual reduction from a zero first
 * guess). */
double orc_residual_norm_zero(orc_hier* H) {
  size_t n = ncells(H, 0);
  double* save = (double*)malloc(n * sizeof(double));
  memcpy(save, H->phi[0], n * sizeof(double));
  memset(H->phi[0], 0, n * sizeof(double));
  double r0 = orc_residual_norm(H);
  memcpy(H->phi[0], save, n * sizeof(double));
  free(save);
  return r0;
}

/* Solve to a relative residual with the run-time order switch of Section 4.
 *
 * order_opt: 0 = automatic switch, 1 = always first order, 2 = always second.
 * Automatic: if the hold counter is positive this solve runs in first order
 * and decrements it.  Otherwise it starts in second order and after every
 * cycle n compares ||r_n|| / ||r_{n-1}|| with eta (r_0 is the residual of the
 * initial guess); above eta it switches to first order for the rest of the
 * solve and sets the hold counter to hold_solves.  Readings where the paper
 * is silent: the test is skipped once ||r_n|| < 100 eps ||r(0)|| (near round
 * off the ratio tends to 1); on a switch the iterate is kept unless its
 * residual exceeds the initial one, in which case the initial guess is
 * restored and the ratio test restarts from it.
 *
 * Stops when ||r_n|| / ||r(Phi=0)|| < tol.  Returns 0 converged, 1 not
 * converged after max_cycles, 2 non-finite residual.  out_info receives
 * {cycles, order at exit, switched, r_zero, r_final, rel}; hist (length
 * max_cycles+1) receives ||r_n||. */
int orc_solve(orc_hier* H, int order_opt, int n_pre, int n_post, int n_cycles, int coarse_sweeps,
              int hold_solves, double eta, double tol, int max_cycles, double* out_info, double* hist) {
  int order = 2, auto_switch = 0, switched = 0;
  if (order_opt == 1) order = 1;
  else if (order_opt == 2) order = 2;
  else if (H->hold > 0) {
    order = 1;
    H->hold -= 1;
  } else {
    auto_switch = 1;
  }
  if (H->deepest[order] < 0) order = 2; /* no first-order hierarchy: cannot happen for level 0 */
  size_t n = ncells(H, 0);
  double r_zero = orc_residual_norm_zero(H);
  double r_init = orc_residual_norm(H);
  double* phi_init = (double*)malloc(n * sizeof(double));
  memcpy(phi_init, H->phi[0], n * sizeof(double));
  if (hist) hist[0] = r_init;
  int status = 1, cycles = 0;
  double r_prev = r_init, r_n = r_init, rel = r_zero > 0 ? r_init / r_zero : 0.0;
  if (!isfinite(r_zero) || !isfinite(r_init)) {
    status = 2; /* non-finite data: nothing to iterate on */
    rel = r_init / r_zero;
  } else if (r_zero == 0.0) {
    memset(H->phi[0], 0, n * sizeof(double));
    r_n = 0.0;
    rel = 0.0;
    status = 0;
  } else if (rel < tol) {
    status = 0;
  } else {
    for (cycles = 1; cycles <= max_cycles; ++cycles) {
      orc_vcycle(H, order, n_pre, n_post, n_cycles, coarse_sweeps);
      r_n = orc_residual_norm(H);
      if (hist) hist[cycles] = r_n;
      if (!isfinite(r_n)) {
        status = 2;
        break;
      }
      rel = r_n / r_zero;
      if (rel < tol) {
        status = 0;
        break;
      }
      if (auto_switch && !switched && order == 2 && r_n >= 100.0 * DBL_EPSILON * r_zero &&
          r_n / r_prev > eta) {
        order = 1;
        switched = 1;
        H->hold = hold_solves;
        if (r_n > r_init) {
          memcpy(H->phi[0], phi_init, n * sizeof(double));
          r_n = r_init;
        }
      }
      r_prev = r_n;
    }
    if (cycles > max_cycles) cycles = max_cycles;
  }
  free(phi_init);
  if (out_info) {
    out_info[0] = cycles;
    out_info[1] = order;
    out_info[2] = switched;
    out_info[3] = r_zero;
    out_info[4] = r_n;
    out_info[5] = rel;
  }
  return status;
}
