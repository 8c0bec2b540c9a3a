/*
 * mw_oracle.c -- plain, slow, FP64 CPU oracle for the mW water model
 * (Molinero & Moore, "Water modeled as an intermediate element between carbon
 * and silicon").
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only code that loads this library.
 * It shares no source, header, table or helper with the CUDA library; the
 * product path never calls it.
 *
 * What it computes, with the passage each part follows:
 *   - Sec. II.A, total energy: E = sum_i sum_{j>i} phi2(r_ij)
 *         + sum_i sum_{j!=i} sum_{k>j} phi3(r_ij, r_ik, theta_jik)
 *     (reading: the angle sits at the centre atom i, both legs start at i,
 *      and every unordered leg pair {j,k} of a centre is counted once).
 *   - Sec. II.A, two-body term:
 *         phi2(r) = A eps [B (sig/r)^p - (sig/r)^q] exp(sig / (r - a sig)),
 *     zero for r >= a sig (reading: the cutoff is a*sig exactly).
 *   - Sec. II.A, three-body term:
 *         phi3 = lam eps [cos th - cos th0]^2 exp(gam sig/(r - a sig))
 *                                          exp(gam sig/(s - a sig)).
 *   - Forces F_i = -dE/dx_i from the analytic derivatives of those terms;
 *     virial W_ab = sum over terms, over the term's legs, of d_a * F_b with
 *     d the leg vector (centre -> partner) and F the force on the partner.
 *   - Sec. II.B: velocity-Verlet dynamics (the paper names LAMMPS, the 10 fs
 *     step and a 1 ps Nose-Hoover relaxation time; the integrator itself and
 *     the single-thermostat Trotter split are this oracle's reading).
 *   - Sec. II.C, structure: the pair histogram behind g(r) (ordered pairs
 *     i != j of one periodic box, binned by their minimum-image distance),
 *     and the angle histogram behind the adf (for each atom k its n_c
 *     nearest neighbours, the angles theta_ikj at k over every ordered pair
 *     i != j of them).  Both by brute force over all pairs.
 *   - Several species (the paper's mW with solutes of their own lambda,
 *     epsilon, sigma, Sec. IV, and the SW family of Fig. 2): the same two
 *     equations with a parameter vector per ordered species triple, in the
 *     usual layout of multi-species SW tables: the pair (i, j) takes the
 *     entry (ti, tj, tj); the three-body term of centre i with legs j, k
 *     takes lambda, epsilon and cos theta0 from (ti, tj, tk), and each leg's
 *     exponential factor (gamma, sigma, a) from that leg's pair entry.  The
 *     paper prints no mixing rule; this is the reading.  Brute force over
 *     all pairs.
 *   - Force-matching adjoint (no counterpart in the paper, whose Sec. II.D
 *     tunes lam, eps, sig by scans): the derivative of the forces along a
 *     direction, taken by the complex-step method (Squire & Trapp, SIAM Rev.
 *     40, 1998), exact to rounding.
 *
 * Two independent force routines are provided: a brute-force O(N^2) pair /
 * O(N^3) triplet enumeration and a cell-list owner loop.  Units are kcal/mol,
 * Angstrom, fs, g/mol, K.
 *
 * Parameter vector layout (double[10]):
 *   0 lambda, 1 epsilon, 2 sigma, 3 a, 4 gamma, 5 A, 6 B, 7 cos_theta0,
 *   8 p, 9 q   (p and q are small non-negative integers stored as doubles).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_KB 0.0019872042586408316 /* kcal/mol/K (R = 8.31446261815324 J/mol/K over 4184 J/kcal) */
#define OR_FCONV 4.184e-4           /* (kcal/mol/A)/(g/mol) expressed in A/fs^2 */

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EOVERFLOW = 3 };

/* ------------------------------------------------------------------ */
/* Parameters (Sec. II.A and Sec. II.D of the paper).                  */
/* ------------------------------------------------------------------ */

void or_params_default(double* prm) {
  prm[0] = 23.15;        /* lambda, Sec. II.D */
  prm[1] = 6.189;        /* epsilon kcal/mol, Sec. II.D */
  prm[2] = 2.3925;       /* sigma Angstrom, Sec. II.D */
  prm[3] = 1.8;          /* a, Sec. II.A */
  prm[4] = 1.2;          /* gamma, Sec. II.A */
  prm[5] = 7.049556277;  /* A, Sec. II.A */
  prm[6] = 0.6022245584; /* B, Sec. II.A */
  prm[7] = -1.0 / 3.0;   /* cos(theta0): tetrahedral angle (reading of 109.47 deg) */
  prm[8] = 4.0;          /* p */
  prm[9] = 0.0;          /* q */
}

/* Threads OpenMP would use (0 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int or_openmp_threads(void) { return omp_get_max_threads(); }
#else
int or_openmp_threads(void) { return 0; }
#endif

static double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

/* phi2(r), Sec. II.A two-body equation. */
double or_phi2(const double* prm, double r) {
  const double eps = prm[1], sig = prm[2], a = prm[3], A = prm[5], B = prm[6];
  const int p = (int)prm[8], q = (int)prm[9];
  if (!(r < a * sig)) return 0.0;
  const double sr = sig / r;
  return A * eps * (B * ipow(sr, p) - ipow(sr, q)) * exp(sig / (r - a * sig));
}

/* d phi2 / dr. */
double or_dphi2(const double* prm, double r) {
  const double eps = prm[1], sig = prm[2], a = prm[3], A = prm[5], B = prm[6];
  const int p = (int)prm[8], q = (int)prm[9];
  if (!(r < a * sig)) return 0.0;
  const double sr = sig / r;
  const double brk = B * ipow(sr, p) - ipow(sr, q);
  const double dbrk = (-p * B * ipow(sr, p) + q * ipow(sr, q)) / r;
  const double x = r - a * sig;
  const double e = exp(sig / x);
  return A * eps * (dbrk * e + brk * e * (-sig / (x * x)));
}

/* phi3(r, s, cos theta), Sec. II.A three-body equation. */
double or_phi3(const double* prm, double r, double s, double cos_t) {
  const double lam = prm[0], eps = prm[1], sig = prm[2], a = prm[3], gam = prm[4], c0 = prm[7];
  if (!(r < a * sig) || !(s < a * sig)) return 0.0;
  const double dc = cos_t - c0;
  return lam * eps * dc * dc * exp(gam * sig / (r - a * sig)) * exp(gam * sig / (s - a * sig));
}

/* phi3 of a centre with leg vectors dj, dk, and its gradient with respect to
 * the two leg vectors (gj = d phi3 / d dj, gk = d phi3 / d dk). */
static double tri_grad(const double* prm, const double* dj, double rj, const double* dk, double rk,
                       double* gj, double* gk) {
  const double lam = prm[0], eps = prm[1], sig = prm[2], a = prm[3], gam = prm[4], c0 = prm[7];
  double uj[3], uk[3];
  for (int d = 0; d < 3; ++d) {
    uj[d] = dj[d] / rj;
    uk[d] = dk[d] / rk;
  }
  const double c = uj[0] * uk[0] + uj[1] * uk[1] + uj[2] * uk[2];
  const double D = c - c0;
  const double xj = rj - a * sig, xk = rk - a * sig;
  const double ej = exp(gam * sig / xj), ek = exp(gam * sig / xk);
  const double pre = lam * eps * ej * ek;
  const double h = pre * D * D;
  const double dlj = -gam * sig / (xj * xj); /* d ln ej / d rj */
  const double dlk = -gam * sig / (xk * xk);
  for (int d = 0; d < 3; ++d) {
    const double dcj = (uk[d] - c * uj[d]) / rj; /* d cos / d dj */
    const double dck = (uj[d] - c * uk[d]) / rk;
    gj[d] = pre * (2.0 * D * dcj + D * D * dlj * uj[d]);
    gk[d] = pre * (2.0 * D * dck + D * D * dlk * uk[d]);
  }
  return h;
}

static void min_image(const double* box, double* d) {
  for (int k = 0; k < 3; ++k) d[k] -= box[k] * nearbyint(d[k] / box[k]);
}

/* virial accumulation: W[xx,yy,zz,xy,xz,yz] += d (x) F; W[6] collects
 * |d_x F_x| + |d_y F_y| + |d_z F_z|, the summed magnitude of the diagonal
 * contributions (the conditioning scale of the trace, which cancels). */
static void add_virial(double* W, const double* d, const double* F) {
  W[6] += fabs(d[0] * F[0]) + fabs(d[1] * F[1]) + fabs(d[2] * F[2]);
  W[0] += d[0] * F[0];
  W[1] += d[1] * F[1];
  W[2] += d[2] * F[2];
  W[3] += d[0] * F[1];
  W[4] += d[0] * F[2];
  W[5] += d[1] * F[2];
}

/*
 * Brute force.  out[0]=E2, out[1]=E3, out[2..7]=W, out[8]=#pairs (r<a sig),
 * out[9]=#triplets (centre, unordered leg pair, both legs < a sig),
 * out[10]=sum over terms and legs of |d_a F_a| (a = x, y, z).
 * f may be NULL.  Requires every box edge >= 2 a sig.
 */
int or_energy_forces_brute(const double* prm, int n, const double* x, const double* box, double* f,
                           double* out) {
  const double rc = prm[3] * prm[2];
  if (n < 0 || box[0] < 2 * rc || box[1] < 2 * rc || box[2] < 2 * rc) return OR_EINVAL;
  double E2 = 0, E3 = 0, W[7] = {0, 0, 0, 0, 0, 0, 0};
  double npair = 0, ntrip = 0;
  if (f) memset(f, 0, sizeof(double) * 3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
      min_image(box, d);
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (!(r < rc)) continue;
      E2 += or_phi2(prm, r);
      const double dp = or_dphi2(prm, r);
      double Fj[3];
      for (int k = 0; k < 3; ++k) Fj[k] = -dp * d[k] / r; /* force on j */
      if (f)
        for (int k = 0; k < 3; ++k) {
          f[3 * j + k] += Fj[k];
          f[3 * i + k] -= Fj[k];
        }
      add_virial(W, d, Fj);
      npair += 1;
    }
  }
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double dj[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
      min_image(box, dj);
      const double rj = sqrt(dj[0] * dj[0] + dj[1] * dj[1] + dj[2] * dj[2]);
      if (!(rj < rc)) continue;
      for (int k = j + 1; k < n; ++k) {
        if (k == i) continue;
        double dk[3] = {x[3 * k] - x[3 * i], x[3 * k + 1] - x[3 * i + 1], x[3 * k + 2] - x[3 * i + 2]};
        min_image(box, dk);
        const double rk = sqrt(dk[0] * dk[0] + dk[1] * dk[1] + dk[2] * dk[2]);
        if (!(rk < rc)) continue;
        double gj[3], gk[3];
        E3 += tri_grad(prm, dj, rj, dk, rk, gj, gk);
        double Fj[3] = {-gj[0], -gj[1], -gj[2]}, Fk[3] = {-gk[0], -gk[1], -gk[2]};
        if (f)
          for (int d = 0; d < 3; ++d) {
            f[3 * j + d] += Fj[d];
            f[3 * k + d] += Fk[d];
            f[3 * i + d] -= Fj[d] + Fk[d];
          }
        add_virial(W, dj, Fj);
        add_virial(W, dk, Fk);
        ntrip += 1;
      }
    }
  }
  out[0] = E2;
  out[1] = E3;
  for (int k = 0; k < 6; ++k) out[2 + k] = W[k];
  out[8] = npair;
  out[9] = ntrip;
  out[10] = W[6];
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Cell list (plain linked cells).                                      */
/* ------------------------------------------------------------------ */

typedef struct {
  int nc[3];
  int* head;
  int* next;
  int* cell_of;
} or_cells;

static double wrap1(double v, double L) {
  double w = v - L * floor(v / L);
  if (w >= L) w -= L;
  if (w < 0) w = 0;
  return w;
}

static int cells_build(or_cells* c, int n, const double* x, const double* box, double rcut) {
  for (int k = 0; k < 3; ++k) {
    c->nc[k] = (int)floor(box[k] / rcut);
    if (c->nc[k] < 1) c->nc[k] = 1;
  }
  const size_t ncell = (size_t)c->nc[0] * c->nc[1] * c->nc[2];
  c->head = (int*)malloc(sizeof(int) * ncell);
  c->next = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  c->cell_of = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!c->head || !c->next || !c->cell_of) return OR_ENOMEM;
  for (size_t i = 0; i < ncell; ++i) c->head[i] = -1;
  /* insert in reverse so each cell lists atoms in ascending index order */
  for (int i = n - 1; i >= 0; --i) {
    int ci[3];
    for (int k = 0; k < 3; ++k) {
      const double w = wrap1(x[3 * i + k], box[k]);
      ci[k] = (int)floor(w / box[k] * c->nc[k]);
      if (ci[k] >= c->nc[k]) ci[k] = c->nc[k] - 1;
      if (ci[k] < 0) ci[k] = 0;
    }
    const int id = (ci[2] * c->nc[1] + ci[1]) * c->nc[0] + ci[0];
    c->cell_of[i] = id;
    c->next[i] = c->head[id];
    c->head[id] = i;
  }
  return OR_OK;
}

static void cells_free(or_cells* c) {
  free(c->head);
  free(c->next);
  free(c->cell_of);
}

/* Distinct cell offsets along one dimension: {-1,0,1} when there are at least
 * three cells, {0,1} for two, {0} for one (so no cell is visited twice). */
static int stencil_offsets(int nc, int* off) {
  if (nc >= 3) {
    off[0] = -1;
    off[1] = 0;
    off[2] = 1;
    return 3;
  }
  if (nc == 2) {
    off[0] = 0;
    off[1] = 1;
    return 2;
  }
  off[0] = 0;
  return 1;
}

/* Gathers the stencil cells around the cell of atom i; returns how many. */
static int stencil_cells(const or_cells* c, int i, int* cells) {
  const int id = c->cell_of[i];
  const int cx = id % c->nc[0], cy = (id / c->nc[0]) % c->nc[1], cz = id / (c->nc[0] * c->nc[1]);
  int ox[3], oy[3], oz[3];
  const int nx = stencil_offsets(c->nc[0], ox), ny = stencil_offsets(c->nc[1], oy),
            nz = stencil_offsets(c->nc[2], oz);
  int m = 0;
  for (int a = 0; a < nz; ++a)
    for (int b = 0; b < ny; ++b)
      for (int g = 0; g < nx; ++g) {
        const int X = (cx + ox[g] + c->nc[0]) % c->nc[0];
        const int Y = (cy + oy[b] + c->nc[1]) % c->nc[1];
        const int Z = (cz + oz[a] + c->nc[2]) % c->nc[2];
        cells[m++] = (Z * c->nc[1] + Y) * c->nc[0] + X;
      }
  return m;
}

typedef struct {
  int j;
  double d[3];
  double r;
} or_leg;

/*
 * Cell-list owner loop.  Same outputs as or_energy_forces_brute.
 * Each atom i gathers its legs (r < a sig); the pair term is taken once per
 * unordered pair (from the lower index), the three-body term once per centre
 * and unordered leg pair.
 */
int or_energy_forces_cell(const double* prm, int n, const double* x, const double* box, double* f,
                          double* out) {
  const double rc = prm[3] * prm[2];
  if (n < 0 || box[0] < 2 * rc || box[1] < 2 * rc || box[2] < 2 * rc) return OR_EINVAL;
  or_cells c;
  if (cells_build(&c, n, x, box, rc) != OR_OK) {
    cells_free(&c);
    return OR_ENOMEM;
  }
  int cap = 64;
  or_leg* legs = (or_leg*)malloc(sizeof(or_leg) * (size_t)cap);
  double E2 = 0, E3 = 0, W[7] = {0, 0, 0, 0, 0, 0, 0};
  double npair = 0, ntrip = 0;
  if (f) memset(f, 0, sizeof(double) * 3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    int cells[27];
    const int ncells = stencil_cells(&c, i, cells);
    int nl = 0;
    for (int s = 0; s < ncells; ++s) {
      for (int j = c.head[cells[s]]; j >= 0; j = c.next[j]) {
        if (j == i) continue;
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(r < rc)) continue;
        if (nl == cap) {
          cap *= 2;
          legs = (or_leg*)realloc(legs, sizeof(or_leg) * (size_t)cap);
        }
        legs[nl].j = j;
        legs[nl].r = r;
        for (int k = 0; k < 3; ++k) legs[nl].d[k] = d[k];
        ++nl;
      }
    }
    for (int l = 0; l < nl; ++l) {
      if (legs[l].j < i) continue;
      const double r = legs[l].r;
      E2 += or_phi2(prm, r);
      const double dp = or_dphi2(prm, r);
      double Fj[3];
      for (int k = 0; k < 3; ++k) Fj[k] = -dp * legs[l].d[k] / r;
      if (f)
        for (int k = 0; k < 3; ++k) {
          f[3 * legs[l].j + k] += Fj[k];
          f[3 * i + k] -= Fj[k];
        }
      add_virial(W, legs[l].d, Fj);
      npair += 1;
    }
    for (int a = 0; a < nl; ++a)
      for (int b = a + 1; b < nl; ++b) {
        double gj[3], gk[3];
        E3 += tri_grad(prm, legs[a].d, legs[a].r, legs[b].d, legs[b].r, gj, gk);
        double Fj[3] = {-gj[0], -gj[1], -gj[2]}, Fk[3] = {-gk[0], -gk[1], -gk[2]};
        if (f)
          for (int d = 0; d < 3; ++d) {
            f[3 * legs[a].j + d] += Fj[d];
            f[3 * legs[b].j + d] += Fk[d];
            f[3 * i + d] -= Fj[d] + Fk[d];
          }
        add_virial(W, legs[a].d, Fj);
        add_virial(W, legs[b].d, Fk);
        ntrip += 1;
      }
  }
  free(legs);
  cells_free(&c);
  out[0] = E2;
  out[1] = E3;
  for (int k = 0; k < 6; ++k) out[2 + k] = W[k];
  out[8] = npair;
  out[9] = ntrip;
  out[10] = W[6];
  return OR_OK;
}

/*
 * Owner-computes variant of or_energy_forces_cell, for the multi-core CPU
 * baseline: the same sums (Sec. II.A), grouped so that every atom's force is
 * assembled by the one thread that owns it, with no shared writes and no
 * atomics.  Pass 1 lists each atom's legs (r < a sig) from the cell list;
 * pass 2 gives atom i
 *   - half of each pair term of its legs (energy, virial) and the pair force
 *     on i;
 *   - the three-body terms centred on i (energy, virial, and their reaction
 *     on i, minus the forces on the two partners);
 *   - the force on i of every three-body term centred on a neighbour j in
 *     which i is one of the two legs (the "two-hop" part: j's legs are read,
 *     nothing of j is written).
 * Same outputs as or_energy_forces_cell (out[8] counts every pair once).
 * nthreads <= 1, or a build without OpenMP, runs serially.
 */
static void add_virial_half(double* W, const double* d, const double* F) {
  double h[3] = {0.5 * F[0], 0.5 * F[1], 0.5 * F[2]};
  add_virial(W, d, h);
}

int or_energy_forces_owner(const double* prm, int n, const double* x, const double* box, double* f, double* out,
                           int nthreads) {
  const double rc = prm[3] * prm[2];
  if (n < 0 || box[0] < 2 * rc || box[1] < 2 * rc || box[2] < 2 * rc) return OR_EINVAL;
  if (nthreads < 1) nthreads = 1;
  or_cells c;
  if (cells_build(&c, n, x, box, rc) != OR_OK) {
    cells_free(&c);
    return OR_ENOMEM;
  }
  int* start = (int*)calloc((size_t)n + 1, sizeof(int));
  if (!start) {
    cells_free(&c);
    return OR_ENOMEM;
  }
  /* pass 1a: leg counts */
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int i = 0; i < n; ++i) {
    int cells[27];
    const int ncells = stencil_cells(&c, i, cells);
    int m = 0;
    for (int s = 0; s < ncells; ++s)
      for (int j = c.head[cells[s]]; j >= 0; j = c.next[j]) {
        if (j == i) continue;
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) < rc) ++m;
      }
    start[i + 1] = m;
  }
  for (int i = 0; i < n; ++i) start[i + 1] += start[i];
  or_leg* legs = (or_leg*)malloc(sizeof(or_leg) * (size_t)(start[n] > 0 ? start[n] : 1));
  if (!legs) {
    free(start);
    cells_free(&c);
    return OR_ENOMEM;
  }
  /* pass 1b: the legs, in stencil order */
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int i = 0; i < n; ++i) {
    int cells[27];
    const int ncells = stencil_cells(&c, i, cells);
    int m = start[i];
    for (int s = 0; s < ncells; ++s)
      for (int j = c.head[cells[s]]; j >= 0; j = c.next[j]) {
        if (j == i) continue;
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(r < rc)) continue;
        legs[m].j = j;
        legs[m].r = r;
        for (int k = 0; k < 3; ++k) legs[m].d[k] = d[k];
        ++m;
      }
  }
  /* pass 2: owner sums */
  double E2 = 0, E3 = 0, W[7] = {0, 0, 0, 0, 0, 0, 0}, npair = 0, ntrip = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 256) reduction(+ : E2, E3, npair, ntrip, W[:7])
  for (int i = 0; i < n; ++i) {
    const or_leg* li = legs + start[i];
    const int nl = start[i + 1] - start[i];
    double Fi[3] = {0, 0, 0};
    for (int l = 0; l < nl; ++l) { /* pair terms, half each side */
      const double r = li[l].r;
      E2 += 0.5 * or_phi2(prm, r);
      const double dp = or_dphi2(prm, r);
      double Fj[3];
      for (int k = 0; k < 3; ++k) Fj[k] = -dp * li[l].d[k] / r;
      for (int k = 0; k < 3; ++k) Fi[k] -= Fj[k];
      add_virial_half(W, li[l].d, Fj);
      npair += 0.5;
    }
    for (int a = 0; a < nl; ++a) /* three-body terms centred on i */
      for (int b = a + 1; b < nl; ++b) {
        double gj[3], gk[3];
        E3 += tri_grad(prm, li[a].d, li[a].r, li[b].d, li[b].r, gj, gk);
        double Fj[3] = {-gj[0], -gj[1], -gj[2]}, Fk[3] = {-gk[0], -gk[1], -gk[2]};
        for (int k = 0; k < 3; ++k) Fi[k] -= Fj[k] + Fk[k];
        add_virial(W, li[a].d, Fj);
        add_virial(W, li[b].d, Fk);
        ntrip += 1;
      }
    for (int l = 0; l < nl; ++l) { /* i as a leg of the terms centred on its neighbour j */
      const int j = li[l].j;
      const or_leg* lj = legs + start[j];
      const int mj = start[j + 1] - start[j];
      int back = -1;
      for (int m = 0; m < mj; ++m)
        if (lj[m].j == i) back = m;
      if (back < 0) continue; /* (cannot happen: the leg relation is symmetric) */
      for (int m = 0; m < mj; ++m) {
        if (m == back) continue;
        double gi[3], gk[3];
        tri_grad(prm, lj[back].d, lj[back].r, lj[m].d, lj[m].r, gi, gk);
        for (int k = 0; k < 3; ++k) Fi[k] -= gi[k];
      }
    }
    if (f)
      for (int k = 0; k < 3; ++k) f[3 * i + k] = Fi[k];
  }
  free(legs);
  free(start);
  cells_free(&c);
  out[0] = E2;
  out[1] = E3;
  for (int k = 0; k < 6; ++k) out[2 + k] = W[k];
  out[8] = npair;
  out[9] = ntrip;
  out[10] = W[6];
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Neighbour sets                                                       */
/* ------------------------------------------------------------------ */

static int cmp_int(const void* a, const void* b) {
  const int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/*
 * For every atom i, the ascending set {j != i : |d_ij|^2 < rlist^2} with d the
 * minimum-image vector.  counts[i] receives the true set size; at most width
 * entries are written to nbr[i*width ...].  Pairs with
 * | |d|^2 - rlist^2 | <= band_rel * rlist^2 are also written (as ordered pairs
 * i, j) to band[] up to band_cap pairs; *nband receives their total number.
 * Returns OR_EOVERFLOW if some set is wider than width (counts stay exact).
 */
int or_neighbors(int n, const double* x, const double* box, double rlist, double band_rel, int width,
                 int* counts, int* nbr, int band_cap, int* band, int* nband) {
  if (n < 0 || box[0] < 2 * rlist || box[1] < 2 * rlist || box[2] < 2 * rlist) return OR_EINVAL;
  or_cells c;
  if (cells_build(&c, n, x, box, rlist) != OR_OK) {
    cells_free(&c);
    return OR_ENOMEM;
  }
  const double rl2 = rlist * rlist;
  int nb = 0, overflow = 0;
  for (int i = 0; i < n; ++i) {
    int cells[27];
    const int ncells = stencil_cells(&c, i, cells);
    int m = 0;
    for (int s = 0; s < ncells; ++s)
      for (int j = c.head[cells[s]]; j >= 0; j = c.next[j]) {
        if (j == i) continue;
        double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
        min_image(box, d);
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (fabs(r2 - rl2) <= band_rel * rl2) {
          if (nb < band_cap) {
            band[2 * nb] = i;
            band[2 * nb + 1] = j;
          }
          ++nb;
        }
        if (r2 < rl2) {
          if (m < width) nbr[(size_t)i * width + m] = j;
          ++m;
        }
      }
    counts[i] = m;
    if (m > width) overflow = 1;
    qsort(nbr + (size_t)i * width, (size_t)(m < width ? m : width), sizeof(int), cmp_int);
  }
  *nband = nb;
  cells_free(&c);
  return overflow ? OR_EOVERFLOW : OR_OK;
}

/* ------------------------------------------------------------------ */
/* Several species.                                                     */
/* ------------------------------------------------------------------ */

/* Entry (a, b, c) of a table of nt^3 parameter vectors. */
static const double* sp_entry(const double* table, int nt, int a, int b, int c) {
  return table + 10 * (((size_t)a * nt + b) * nt + c);
}

/* The table's own consistency: the pair term of (a, b) must not depend on
 * which of the two is taken first, and the three-body term of a centre a
 * must not depend on the order of its legs b, c. */
int or_species_table_check(const double* table, int nt) {
  if (nt < 1) return OR_EINVAL;
  static const int pair_fields[] = {1, 2, 3, 5, 6, 8, 9};
  static const int tri_fields[] = {0, 1, 7};
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const double* ab = sp_entry(table, nt, a, b, b);
      const double* ba = sp_entry(table, nt, b, a, a);
      for (int k = 0; k < 7; ++k)
        if (ab[pair_fields[k]] != ba[pair_fields[k]]) return OR_EINVAL;
      if (!(ab[2] > 0) || !(ab[3] > 0)) return OR_EINVAL;
      for (int c = 0; c < nt; ++c) {
        const double* abc = sp_entry(table, nt, a, b, c);
        const double* acb = sp_entry(table, nt, a, c, b);
        for (int k = 0; k < 3; ++k)
          if (abc[tri_fields[k]] != acb[tri_fields[k]]) return OR_EINVAL;
      }
    }
  return OR_OK;
}

/* Three-body term of a centre whose legs carry their own exponential
 * factors: lam eps (cos - c0)^2 exp(gj sj/(rj - aj sj)) exp(gk sk/(rk - ak sk)),
 * with lam, eps, c0 from pt and (gamma, sigma, a) of each leg from pj, pk;
 * gradient with respect to the two leg vectors as in tri_grad. */
static double sp_tri_grad(const double* pt, const double* pj, const double* pk, const double* dj, double rj,
                          const double* dk, double rk, double* gj, double* gk) {
  const double lam = pt[0], eps = pt[1], c0 = pt[7];
  const double sj = pj[2], aj = pj[3], gmj = pj[4];
  const double sk = pk[2], ak = pk[3], gmk = pk[4];
  double uj[3], uk[3];
  for (int d = 0; d < 3; ++d) {
    uj[d] = dj[d] / rj;
    uk[d] = dk[d] / rk;
  }
  const double c = uj[0] * uk[0] + uj[1] * uk[1] + uj[2] * uk[2];
  const double D = c - c0;
  const double xj = rj - aj * sj, xk = rk - ak * sk;
  const double pre = lam * eps * exp(gmj * sj / xj) * exp(gmk * sk / xk);
  const double dlj = -gmj * sj / (xj * xj);
  const double dlk = -gmk * sk / (xk * xk);
  for (int d = 0; d < 3; ++d) {
    const double dcj = (uk[d] - c * uj[d]) / rj;
    const double dck = (uj[d] - c * uk[d]) / rk;
    gj[d] = pre * (2.0 * D * dcj + D * D * dlj * uj[d]);
    gk[d] = pre * (2.0 * D * dck + D * D * dlk * uk[d]);
  }
  return pre * D * D;
}

/*
 * Energy, forces and virial of a box of several species, by brute force.
 * table: nt^3 parameter vectors (layout of or_params_default), entry
 * (a, b, c) at index (a nt + b) nt + c; types[n] in [0, nt).  Outputs as
 * or_energy_forces_brute (out[8] pairs, out[9] triplets).  Requires every
 * edge >= 2 max(a sigma).
 */
int or_energy_forces_species(const double* table, int nt, const int* types, int n, const double* x,
                             const double* box, double* f, double* out) {
  if (n < 0 || or_species_table_check(table, nt) != OR_OK) return OR_EINVAL;
  double rcmax = 0;
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const double* e = sp_entry(table, nt, a, b, b);
      if (e[3] * e[2] > rcmax) rcmax = e[3] * e[2];
    }
  if (box[0] < 2 * rcmax || box[1] < 2 * rcmax || box[2] < 2 * rcmax) return OR_EINVAL;
  for (int i = 0; i < n; ++i)
    if (types[i] < 0 || types[i] >= nt) return OR_EINVAL;
  double E2 = 0, E3 = 0, W[7] = {0, 0, 0, 0, 0, 0, 0};
  double npair = 0, ntrip = 0;
  if (f) memset(f, 0, sizeof(double) * 3 * (size_t)n);
  int cap = 64;
  or_leg* legs = (or_leg*)malloc(sizeof(or_leg) * (size_t)cap);
  if (!legs) return OR_ENOMEM;
  for (int i = 0; i < n; ++i) {
    const int ti = types[i];
    int nl = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double* pij = sp_entry(table, nt, ti, types[j], types[j]);
      double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
      min_image(box, d);
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (!(r < pij[3] * pij[2])) continue;
      if (nl == cap) {
        cap *= 2;
        or_leg* nlg = (or_leg*)realloc(legs, sizeof(or_leg) * (size_t)cap);
        if (!nlg) {
          free(legs);
          return OR_ENOMEM;
        }
        legs = nlg;
      }
      legs[nl].j = j;
      legs[nl].r = r;
      for (int k = 0; k < 3; ++k) legs[nl].d[k] = d[k];
      ++nl;
      if (j > i) { /* pair term once per unordered pair */
        E2 += or_phi2(pij, r);
        const double dp = or_dphi2(pij, r);
        double Fj[3];
        for (int k = 0; k < 3; ++k) Fj[k] = -dp * d[k] / r;
        if (f)
          for (int k = 0; k < 3; ++k) {
            f[3 * j + k] += Fj[k];
            f[3 * i + k] -= Fj[k];
          }
        add_virial(W, d, Fj);
        npair += 1;
      }
    }
    for (int a = 0; a < nl; ++a)
      for (int b = a + 1; b < nl; ++b) {
        const int tj = types[legs[a].j], tk = types[legs[b].j];
        double gj[3], gk[3];
        E3 += sp_tri_grad(sp_entry(table, nt, ti, tj, tk), sp_entry(table, nt, ti, tj, tj),
                          sp_entry(table, nt, ti, tk, tk), legs[a].d, legs[a].r, legs[b].d, legs[b].r, gj, gk);
        double Fj[3] = {-gj[0], -gj[1], -gj[2]}, Fk[3] = {-gk[0], -gk[1], -gk[2]};
        if (f)
          for (int d = 0; d < 3; ++d) {
            f[3 * legs[a].j + d] += Fj[d];
            f[3 * legs[b].j + d] += Fk[d];
            f[3 * i + d] -= Fj[d] + Fk[d];
          }
        add_virial(W, legs[a].d, Fj);
        add_virial(W, legs[b].d, Fk);
        ntrip += 1;
      }
  }
  free(legs);
  out[0] = E2;
  out[1] = E3;
  for (int k = 0; k < 6; ++k) out[2 + k] = W[k];
  out[8] = npair;
  out[9] = ntrip;
  out[10] = W[6];
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Dynamics: velocity Verlet with an optional thermostat (Sec. II.B).   */
/* ------------------------------------------------------------------ */

static double kinetic(int n, const double* v, double mass) {
  double s = 0;
  for (int i = 0; i < 3 * n; ++i) s += v[i] * v[i];
  return 0.5 * mass * s / OR_FCONV; /* kcal/mol */
}

/* kinetic() summed by nt threads (the multi-core baseline; nt <= 1 is kinetic()). */
static double kinetic_nt(int n, const double* v, double mass, int nt) {
  if (nt <= 1) return kinetic(n, v, mass);
  double s = 0;
#pragma omp parallel for num_threads(nt) schedule(static) reduction(+ : s)
  for (int i = 0; i < 3 * n; ++i) s += v[i] * v[i];
  return 0.5 * mass * s / OR_FCONV;
}

/* One Nose-Hoover half step (length dt/2) of a single thermostat, split as
 * quarter step on xi, velocity scaling, half step on eta, quarter step on xi.
 * Q = Ndf kB T0 tau^2. */
static void nh_half(int n, double* v, double* ke, double* xi, double* eta, double dt, double Ndf, double T0,
                    double Q) {
  double G = (2.0 * (*ke) - Ndf * OR_KB * T0) / Q;
  *xi += 0.25 * dt * G;
  const double s = exp(-(*xi) * 0.5 * dt);
  for (int i = 0; i < 3 * n; ++i) v[i] *= s;
  *ke *= s * s;
  *eta += (*xi) * 0.5 * dt;
  G = (2.0 * (*ke) - Ndf * OR_KB * T0) / Q;
  *xi += 0.25 * dt * G;
}

/*
 * Runs nsteps velocity-Verlet steps in place on x, v (n*3, A and A/fs).
 * kind: 0 NVE, 1 Berendsen (v scaled by sqrt(1 + dt/tau (T0/T - 1)) after
 * each step), 2 Nose-Hoover (symmetric Trotter split around the Verlet step).
 * state[0] = xi (1/fs), state[1] = eta (dimensionless), updated in place.
 * thermo (nsteps+1)*8 doubles, may be NULL: per step (index 0 = initial)
 *   pe, e2, e3, ke, T, conserved, xi, eta
 * conserved = ke + pe (+ Q xi^2 / 2 + Ndf kB T0 eta under Nose-Hoover).
 * Positions are wrapped into [0, L).  Ndf = 3n - 3.
 */
typedef struct {
  const double* prm; /* one species: parameter vector */
  const double* table; /* several species: nt^3 vectors, or NULL */
  int nt;
  const int* types;
  int nthreads; /* > 0: one species through or_energy_forces_owner on that many threads */
} md_pot;

static int md_forces(const md_pot* pot, int n, const double* x, const double* box, double* f, double* out) {
  if (pot->table) return or_energy_forces_species(pot->table, pot->nt, pot->types, n, x, box, f, out);
  if (pot->nthreads > 0) return or_energy_forces_owner(pot->prm, n, x, box, f, out, pot->nthreads);
  return or_energy_forces_cell(pot->prm, n, x, box, f, out);
}

static int md_run(const md_pot* pot, int n, double* x, double* v, const double* box, double mass, double dt,
                  int kind, double T0, double tau, int nsteps, double* state, double* thermo);

int or_md(const double* prm, int n, double* x, double* v, const double* box, double mass, double dt,
          int kind, double T0, double tau, int nsteps, double* state, double* thermo) {
  const md_pot pot = {prm, NULL, 0, NULL, 0};
  return md_run(&pot, n, x, v, box, mass, dt, kind, T0, tau, nsteps, state, thermo);
}

/* or_md with the owner-computes forces on nthreads threads (the multi-core
 * CPU baseline); the same trajectory as or_md up to rounding order. */
int or_md_owner(const double* prm, int n, double* x, double* v, const double* box, double mass, double dt,
                int kind, double T0, double tau, int nsteps, double* state, double* thermo, int nthreads) {
  const md_pot pot = {prm, NULL, 0, NULL, nthreads > 0 ? nthreads : 1};
  return md_run(&pot, n, x, v, box, mass, dt, kind, T0, tau, nsteps, state, thermo);
}

/* or_md with the several-species potential of or_energy_forces_species. */
int or_md_species(const double* table, int nt, const int* types, int n, double* x, double* v, const double* box,
                  double mass, double dt, int kind, double T0, double tau, int nsteps, double* state,
                  double* thermo) {
  const md_pot pot = {NULL, table, nt, types, 0};
  return md_run(&pot, n, x, v, box, mass, dt, kind, T0, tau, nsteps, state, thermo);
}

static int md_run(const md_pot* pot, int n, double* x, double* v, const double* box, double mass, double dt,
                  int kind, double T0, double tau, int nsteps, double* state, double* thermo) {
  if (n < 2 || kind < 0 || kind > 2) return OR_EINVAL;
  double* f = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  if (!f) return OR_ENOMEM;
  double out[11];
  for (int i = 0; i < 3 * n; ++i) x[i] = wrap1(x[i], box[i % 3]);
  int rc = md_forces(pot, n, x, box, f, out);
  if (rc != OR_OK) {
    free(f);
    return rc;
  }
  const double Ndf = 3.0 * n - 3.0;
  const double Q = Ndf * OR_KB * T0 * tau * tau;
  double xi = state[0], eta = state[1];
  const double cf = 0.5 * dt * OR_FCONV / mass;
  const int nt = pot->nthreads;
  for (int s = 0; s <= nsteps; ++s) {
    if (s > 0) {
      double ke = kinetic_nt(n, v, mass, nt);
      if (kind == 2) nh_half(n, v, &ke, &xi, &eta, dt, Ndf, T0, Q);
#pragma omp parallel for if (nt > 1) num_threads(nt > 1 ? nt : 1) schedule(static)
      for (int i = 0; i < 3 * n; ++i) {
        v[i] += cf * f[i];
        x[i] = wrap1(x[i] + dt * v[i], box[i % 3]);
      }
      rc = md_forces(pot, n, x, box, f, out);
      if (rc != OR_OK) break;
#pragma omp parallel for if (nt > 1) num_threads(nt > 1 ? nt : 1) schedule(static)
      for (int i = 0; i < 3 * n; ++i) v[i] += cf * f[i];
      ke = kinetic_nt(n, v, mass, nt);
      if (kind == 2) nh_half(n, v, &ke, &xi, &eta, dt, Ndf, T0, Q);
      if (kind == 1) {
        const double T = 2.0 * ke / (Ndf * OR_KB);
        const double lam = sqrt(1.0 + dt / tau * (T0 / T - 1.0));
        for (int i = 0; i < 3 * n; ++i) v[i] *= lam;
      }
    }
    if (thermo) {
      const double ke = kinetic(n, v, mass);
      const double pe = out[0] + out[1];
      double cons = ke + pe;
      if (kind == 2) cons += 0.5 * Q * xi * xi + Ndf * OR_KB * T0 * eta;
      double* t = thermo + 8 * (size_t)s;
      t[0] = pe;
      t[1] = out[0];
      t[2] = out[1];
      t[3] = ke;
      t[4] = 2.0 * ke / (Ndf * OR_KB);
      t[5] = cons;
      t[6] = xi;
      t[7] = eta;
    }
  }
  state[0] = xi;
  state[1] = eta;
  free(f);
  return rc;
}

/*
 * Isobaric-isothermal dynamics.  Sec. II.B controls pressure with a
 * Nose-Hoover barostat (relaxation time 2.5 ps, p = 0) next to the 1 ps
 * Nose-Hoover thermostat; read as the isotropic Martyna-Tobias-Klein
 * equations with the single particle thermostat of or_md:
 *   dr/dt = v + (pe/W) r,   dv/dt = F/m - (1 + 3/Ndf) (pe/W) v - xi v,
 *   dL/dt = (pe/W) L,       dpe/dt = (1 + 3/Ndf) 2 KE + tr(Wv) - 3 P V,
 * W = (Ndf + 3) kB T0 tau_p^2, Wv the virial (sum over legs of d F), V = Lx Ly Lz.
 * Symmetric Trotter split per step: thermostat half; barostat half on pe;
 * friction half (v times exp(-dt/2 (1 + 3/Ndf) pe/W)); kick; drift
 * r -> r e^u + v dt e^(u/2) sinh(u/2)/(u/2), L -> L e^u with u = dt pe/W;
 * forces; kick; friction half; barostat half; thermostat half.
 * P in kcal/mol/A^3.  box[3] is scaled in place; state = xi, eta, pe.
 * thermo (nsteps+1)*10, may be NULL: pe, e2, e3, ke, T, conserved, xi, eta,
 * V, pressure (kcal/mol/A^3); conserved = ke + pe + P V + pe^2/(2W)
 *   + Q xi^2/2 + Ndf kB T0 eta.  Positions are wrapped into [0, L).
 */
static int npt_run(const md_pot* pot, int n, double* x, double* v, double* box, double mass, double dt, double T0,
                   double tau, double P, double tau_p, int nsteps, double* state, double* thermo);

int or_md_npt(const double* prm, int n, double* x, double* v, double* box, double mass, double dt, double T0,
              double tau, double P, double tau_p, int nsteps, double* state, double* thermo) {
  const md_pot pot = {prm, NULL, 0, NULL, 0};
  return npt_run(&pot, n, x, v, box, mass, dt, T0, tau, P, tau_p, nsteps, state, thermo);
}

/* or_md_npt with the several-species potential of or_energy_forces_species. */
int or_md_npt_species(const double* table, int nt, const int* types, int n, double* x, double* v, double* box,
                      double mass, double dt, double T0, double tau, double P, double tau_p, int nsteps,
                      double* state, double* thermo) {
  const md_pot pot = {NULL, table, nt, types, 0};
  return npt_run(&pot, n, x, v, box, mass, dt, T0, tau, P, tau_p, nsteps, state, thermo);
}

static int npt_run(const md_pot* pot, int n, double* x, double* v, double* box, double mass, double dt, double T0,
                   double tau, double P, double tau_p, int nsteps, double* state, double* thermo) {
  if (n < 2) return OR_EINVAL;
  double* f = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  if (!f) return OR_ENOMEM;
  double out[11];
  for (int i = 0; i < 3 * n; ++i) x[i] = wrap1(x[i], box[i % 3]);
  int rc = md_forces(pot, n, x, box, f, out);
  if (rc != OR_OK) {
    free(f);
    return rc;
  }
  const double Ndf = 3.0 * n - 3.0;
  const double Q = Ndf * OR_KB * T0 * tau * tau;
  const double W = (Ndf + 3.0) * OR_KB * T0 * tau_p * tau_p;
  const double a3 = 1.0 + 3.0 / Ndf;
  double xi = state[0], eta = state[1], pe = state[2];
  const double cf = 0.5 * dt * OR_FCONV / mass;
  for (int s = 0; s <= nsteps; ++s) {
    if (s > 0) {
      double ke = kinetic(n, v, mass);
      double V = box[0] * box[1] * box[2];
      nh_half(n, v, &ke, &xi, &eta, dt, Ndf, T0, Q);
      pe += 0.5 * dt * (a3 * 2.0 * ke + (out[2] + out[3] + out[4]) - 3.0 * P * V);
      const double fr = exp(-0.5 * dt * a3 * pe / W);
      for (int i = 0; i < 3 * n; ++i) v[i] *= fr;
      for (int i = 0; i < 3 * n; ++i) v[i] += cf * f[i];
      const double u = dt * pe / W;
      const double eu = exp(u);
      const double sh = (fabs(u) > 1e-8) ? exp(0.5 * u) * sinh(0.5 * u) / (0.5 * u) : 1.0 + 0.5 * u;
      for (int k = 0; k < 3; ++k) box[k] *= eu;
      for (int i = 0; i < 3 * n; ++i) x[i] = wrap1(x[i] * eu + v[i] * dt * sh, box[i % 3]);
      rc = md_forces(pot, n, x, box, f, out);
      if (rc != OR_OK) break;
      for (int i = 0; i < 3 * n; ++i) v[i] += cf * f[i];
      for (int i = 0; i < 3 * n; ++i) v[i] *= fr;  /* pe is unchanged since the first friction half */
      ke = kinetic(n, v, mass);
      V = box[0] * box[1] * box[2];
      pe += 0.5 * dt * (a3 * 2.0 * ke + (out[2] + out[3] + out[4]) - 3.0 * P * V);
      nh_half(n, v, &ke, &xi, &eta, dt, Ndf, T0, Q);
    }
    if (thermo) {
      const double ke = kinetic(n, v, mass);
      const double epot = out[0] + out[1];
      const double V = box[0] * box[1] * box[2];
      double* t = thermo + 10 * (size_t)s;
      t[0] = epot;
      t[1] = out[0];
      t[2] = out[1];
      t[3] = ke;
      t[4] = 2.0 * ke / (Ndf * OR_KB);
      t[5] = ke + epot + P * V + 0.5 * pe * pe / W + 0.5 * Q * xi * xi + Ndf * OR_KB * T0 * eta;
      t[6] = xi;
      t[7] = eta;
      t[8] = V;
      t[9] = (2.0 * ke + out[2] + out[3] + out[4]) / (3.0 * V);
    }
  }
  state[0] = xi;
  state[1] = eta;
  state[2] = pe;
  free(f);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Complex-step derivatives for the force-matching adjoint.             */
/* ------------------------------------------------------------------ */

typedef double complex cplx;

static cplx cipow(cplx x, int n) {
  cplx r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

/*
 * The same cell-list energy and forces as or_energy_forces_cell, evaluated in
 * complex arithmetic with complex parameters pc[0..7] and complex positions
 * xc.  Branches (cutoff, minimum image, cell membership) use real parts.
 * energy_out may be NULL.
 */
static int cs_energy_forces(const cplx* pc, const double* prm_real, int n, const cplx* xc, const double* box,
                            cplx* f, cplx* energy_out) {
  const cplx lam = pc[0], eps = pc[1], sig = pc[2], a = pc[3], gam = pc[4], A = pc[5], B = pc[6], c0 = pc[7];
  const int p = (int)prm_real[8], q = (int)prm_real[9];
  const double rc_real = creal(a * sig);
  double* xr = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  if (!xr) return OR_ENOMEM;
  for (int i = 0; i < 3 * n; ++i) xr[i] = creal(xc[i]);
  or_cells c;
  if (cells_build(&c, n, xr, box, rc_real) != OR_OK) {
    cells_free(&c);
    free(xr);
    return OR_ENOMEM;
  }
  int cap = 64;
  int* lj = (int*)malloc(sizeof(int) * (size_t)cap);
  cplx* ld = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)cap);
  cplx* lr = (cplx*)malloc(sizeof(cplx) * (size_t)cap);
  for (int i = 0; i < 3 * n; ++i) f[i] = 0;
  cplx E = 0;
  for (int i = 0; i < n; ++i) {
    int cells[27];
    const int ncells = stencil_cells(&c, i, cells);
    int nl = 0;
    for (int s = 0; s < ncells; ++s)
      for (int j = c.head[cells[s]]; j >= 0; j = c.next[j]) {
        if (j == i) continue;
        cplx d[3];
        for (int k = 0; k < 3; ++k) {
          d[k] = xc[3 * j + k] - xc[3 * i + k];
          d[k] -= box[k] * nearbyint(creal(d[k]) / box[k]);
        }
        const cplx r = csqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(creal(r) < rc_real)) continue;
        if (nl == cap) {
          cap *= 2;
          lj = (int*)realloc(lj, sizeof(int) * (size_t)cap);
          ld = (cplx*)realloc(ld, sizeof(cplx) * 3 * (size_t)cap);
          lr = (cplx*)realloc(lr, sizeof(cplx) * (size_t)cap);
        }
        lj[nl] = j;
        lr[nl] = r;
        for (int k = 0; k < 3; ++k) ld[3 * nl + k] = d[k];
        ++nl;
      }
    /* pair terms, once per unordered pair */
    for (int l = 0; l < nl; ++l) {
      if (lj[l] < i) continue;
      const cplx r = lr[l];
      const cplx sr = sig / r;
      const cplx brk = B * cipow(sr, p) - cipow(sr, q);
      const cplx dbrk = (-(double)p * B * cipow(sr, p) + (double)q * cipow(sr, q)) / r;
      const cplx xx = r - a * sig;
      const cplx e = cexp(sig / xx);
      E += A * eps * brk * e;
      const cplx dp = A * eps * (dbrk * e + brk * e * (-sig / (xx * xx)));
      for (int k = 0; k < 3; ++k) {
        const cplx Fj = -dp * ld[3 * l + k] / r;
        f[3 * lj[l] + k] += Fj;
        f[3 * i + k] -= Fj;
      }
    }
    /* three-body terms, once per centre and unordered leg pair */
    for (int u = 0; u < nl; ++u)
      for (int w = u + 1; w < nl; ++w) {
        const cplx rj = lr[u], rk = lr[w];
        cplx uj[3], uk[3];
        for (int k = 0; k < 3; ++k) {
          uj[k] = ld[3 * u + k] / rj;
          uk[k] = ld[3 * w + k] / rk;
        }
        const cplx cth = uj[0] * uk[0] + uj[1] * uk[1] + uj[2] * uk[2];
        const cplx D = cth - c0;
        const cplx xj = rj - a * sig, xk = rk - a * sig;
        const cplx ej = cexp(gam * sig / xj), ek = cexp(gam * sig / xk);
        const cplx pre = lam * eps * ej * ek;
        E += pre * D * D;
        const cplx dlj = -gam * sig / (xj * xj), dlk = -gam * sig / (xk * xk);
        for (int k = 0; k < 3; ++k) {
          const cplx gj = pre * (2.0 * D * (uk[k] - cth * uj[k]) / rj + D * D * dlj * uj[k]);
          const cplx gk = pre * (2.0 * D * (uj[k] - cth * uk[k]) / rk + D * D * dlk * uk[k]);
          f[3 * lj[u] + k] -= gj;
          f[3 * lj[w] + k] -= gk;
          f[3 * i + k] += gj + gk;
        }
      }
  }
  free(lj);
  free(ld);
  free(lr);
  cells_free(&c);
  free(xr);
  if (energy_out) *energy_out = E;
  return OR_OK;
}

/*
 * Adjoint of the forces.  Given w = dL/dF (n*3), returns
 *   dLdx[m]      = sum_i w_i . dF_i/dx_m        (n*3)
 *   dLdtheta[0..2] = sum_i w_i . dF_i/d(lambda, epsilon, sigma)
 * Each is one complex-step directional derivative: F(x + i h w) gives
 * (dF/dx) w, which equals the row contraction w^T (dF/dx) because dF/dx is
 * minus the (symmetric) Hessian of E; F(theta_p + i h) gives dF/dtheta_p.
 */
int or_force_vjp(const double* prm, int n, const double* x, const double* box, const double* w, double* dLdx,
                 double* dLdtheta) {
  if (n < 1) return OR_EINVAL;
  const double h = 1e-30;
  double wmax = 0;
  for (int i = 0; i < 3 * n; ++i) wmax = fmax(wmax, fabs(w[i]));
  cplx pc[8];
  cplx* xc = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)n);
  cplx* fc = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)n);
  if (!xc || !fc) {
    free(xc);
    free(fc);
    return OR_ENOMEM;
  }
  int rc = OR_OK;
  for (int k = 0; k < 8; ++k) pc[k] = prm[k];
  if (dLdx) {
    if (wmax == 0) {
      memset(dLdx, 0, sizeof(double) * 3 * (size_t)n);
    } else {
      for (int i = 0; i < 3 * n; ++i) xc[i] = x[i] + I * h * (w[i] / wmax);
      rc = cs_energy_forces(pc, prm, n, xc, box, fc, NULL);
      for (int i = 0; i < 3 * n; ++i) dLdx[i] = cimag(fc[i]) / h * wmax;
    }
  }
  if (dLdtheta && rc == OR_OK) {
    for (int i = 0; i < 3 * n; ++i) xc[i] = x[i];
    for (int t = 0; t < 3 && rc == OR_OK; ++t) {
      for (int k = 0; k < 8; ++k) pc[k] = prm[k];
      pc[t] += I * h;
      rc = cs_energy_forces(pc, prm, n, xc, box, fc, NULL);
      double s = 0;
      for (int i = 0; i < 3 * n; ++i) s += w[i] * (cimag(fc[i]) / h);
      dLdtheta[t] = s;
    }
  }
  free(xc);
  free(fc);
  return rc;
}

/* dE/d(lambda, epsilon, sigma) by complex step on the energy. */
int or_energy_param_grad(const double* prm, int n, const double* x, const double* box, double* dEdtheta) {
  const double h = 1e-30;
  cplx pc[8];
  cplx* xc = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)n);
  cplx* fc = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)n);
  if (!xc || !fc) {
    free(xc);
    free(fc);
    return OR_ENOMEM;
  }
  for (int i = 0; i < 3 * n; ++i) xc[i] = x[i];
  int rc = OR_OK;
  for (int t = 0; t < 3 && rc == OR_OK; ++t) {
    for (int k = 0; k < 8; ++k) pc[k] = prm[k];
    pc[t] += I * h;
    cplx E;
    rc = cs_energy_forces(pc, prm, n, xc, box, fc, &E);
    dEdtheta[t] = cimag(E) / h;
  }
  free(xc);
  free(fc);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Sec. II.C, structure.
 *
 * Pair histogram: hist[k] = number of ordered pairs (i, j), i != j, whose
 * minimum-image distance r satisfies k dr <= r < (k + 1) dr, k < nbins.
 * amb[k] counts the pairs whose r lies within rel * r of a bin edge of bin k
 * (the bin a rounding of r could move them into or out of).  All pairs by
 * brute force.  Returns 0. */
int or_pair_histogram(int n, const double* x, const double* box, double dr, int nbins, double rel, long long* hist,
                      long long* amb) {
  for (int k = 0; k < nbins; ++k) hist[k] = amb[k] = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
      min_image(box, d);
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      const double t = r / dr;
      const int k = (int)floor(t);
      if (k >= 0 && k < nbins) hist[k] += 1;
      /* near an edge: count in both neighbouring bins */
      const double e = floor(t + 0.5);
      if (fabs(t - e) * dr <= rel * r) {
        const int lo = (int)e - 1, hi = (int)e;
        if (lo >= 0 && lo < nbins) amb[lo] += 1;
        if (hi >= 0 && hi < nbins) amb[hi] += 1;
      }
    }
  return 0;
}

typedef struct {
  double r2;
  int j;
} or_nb;

static int cmp_nb(const void* a, const void* b) {
  const or_nb* p = (const or_nb*)a;
  const or_nb* q = (const or_nb*)b;
  if (p->r2 < q->r2) return -1;
  if (p->r2 > q->r2) return 1;
  return (p->j > q->j) - (p->j < q->j);
}

/* Angle histogram (adf): for each atom k, its nc nearest neighbours (ties by
 * index); for every ordered pair (i, j), i != j, of them the angle theta_ikj
 * at k, binned over [0, 180] degrees in nbins bins (180 itself in the last).
 * amb[b] counts the angles within tol_deg of an edge of bin b; *ties counts
 * the atoms whose nc-th and (nc+1)-th neighbour distances differ by less than
 * rel of the distance (the selection a rounding could change).  Returns 0,
 * or -1 if an atom has fewer than nc other atoms. */
int or_angle_histogram(int n, const double* x, const double* box, int nc, int nbins, double tol_deg, double rel,
                       long long* hist, long long* amb, long long* ties) {
  const double pi = 3.14159265358979323846;
  const double w = 180.0 / nbins;
  for (int b = 0; b < nbins; ++b) hist[b] = amb[b] = 0;
  *ties = 0;
  if (nc >= n) return -1;
  or_nb* nb = (or_nb*)malloc(sizeof(or_nb) * (size_t)n);
  double* u = (double*)malloc(sizeof(double) * 3 * (size_t)nc);
  if (!nb || !u) {
    free(nb);
    free(u);
    return -2;
  }
  for (int k = 0; k < n; ++k) {
    int m = 0;
    for (int j = 0; j < n; ++j) {
      if (j == k) continue;
      double d[3] = {x[3 * j] - x[3 * k], x[3 * j + 1] - x[3 * k + 1], x[3 * j + 2] - x[3 * k + 2]};
      min_image(box, d);
      nb[m].r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      nb[m].j = j;
      ++m;
    }
    qsort(nb, (size_t)m, sizeof(or_nb), cmp_nb);
    if (m > nc) {
      const double ra = sqrt(nb[nc - 1].r2), rb = sqrt(nb[nc].r2);
      if (rb - ra <= rel * rb) *ties += 1;
    }
    for (int a = 0; a < nc; ++a) {
      const int j = nb[a].j;
      double d[3] = {x[3 * j] - x[3 * k], x[3 * j + 1] - x[3 * k + 1], x[3 * j + 2] - x[3 * k + 2]};
      min_image(box, d);
      const double r = sqrt(nb[a].r2);
      for (int c = 0; c < 3; ++c) u[3 * a + c] = d[c] / r;
    }
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b) {
        if (a == b) continue;
        double c = u[3 * a] * u[3 * b] + u[3 * a + 1] * u[3 * b + 1] + u[3 * a + 2] * u[3 * b + 2];
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        const double th = acos(c) * 180.0 / pi;
        int bin = (int)floor(th / w);
        if (bin >= nbins) bin = nbins - 1;
        if (bin < 0) bin = 0;
        hist[bin] += 1;
        const double e = floor(th / w + 0.5);
        if (fabs(th - e * w) <= tol_deg) {
          const int lo = (int)e - 1, hi = (int)e;
          if (lo >= 0 && lo < nbins) amb[lo] += 1;
          if (hi >= 0 && hi < nbins) amb[hi] += 1;
        }
      }
  }
  free(nb);
  free(u);
  return 0;
}
