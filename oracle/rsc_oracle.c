/*
 * rsc_oracle.c -- plain FP64 CPU oracle for rotational orthogonal matching
 * pursuit (rotational OMP) in a steerable circular-harmonic basis.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library; the two sides meet only through the seeded inputs.
 *
 * What it computes (McCann et al., "Fast Rotational Sparse Coding"):
 *   - Problem: Eq. (rot-SC) in Sec. II-B -- each patch x is coded by at most K
 *     (atom m, angle index r, weight a) triples, atom m rotated by 2*pi*r/R.
 *   - Rotation in the steerable basis is the diagonal steering matrix of
 *     Eq. (Sr), Sec. II-D: harmonic t of a coefficient vector is multiplied by
 *     exp(-i t 2 pi r / R) (read off Eq. (rotation)).
 *   - After the change of basis of Eq. (rearrange) the whole objective lives
 *     in coefficient space, where the inner product is the plain complex one.
 *   - The coder is OMP (Sec. II-C, the OMP call in the R-K-SVD pseudocode of
 *     Fig. "code") run on the augmented dictionary [S_0 D, ..., S_{R-1} D],
 *     which this oracle materialises explicitly, as Fig. "code" does.
 *
 * Steps follow the paper's order and notation, deliberately without any of
 * the GPU path's factorisations:
 *   1. expand each stored half spectrum (harmonics k = 0..kmax) to the full
 *      spectrum k = -kmax..kmax using Hermitian symmetry of a real patch
 *      (c[j,-k] = conj(c[j,k]); the k = 0 entry is real);
 *   2. materialise every steered atom A_{m,r} = S_r d_m;
 *   3. OMP: score every A_{m,r} against the residual, take the largest
 *      |score| (ties: smallest flat index m*R + r), rebuild the Gram matrix of
 *      the selected steered atoms from scratch, solve the least-squares
 *      problem by Cholesky, recompute the residual x - sum_i a_i A_i.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - selection uses |<A, r>| (OMP with unit-norm atoms, weights of any sign);
 *   - coefficients are real (real patches, Hermitian spectra);
 *   - a step stops the coding of a patch when max |score| <= STOP_REL * ||x||
 *     or when the new Cholesky pivot^2 <= PIVOT_REL * Gram diagonal entry; the
 *     remaining outputs are atom = angle = -1, coefficient 0.
 *
 * Layout of the half spectra (input): [k][j][re,im] floats, k = 0..kmax,
 * j = 0..J-1, so one patch / atom is (kmax+1)*J*2 floats; Im of k = 0 is
 * ignored.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define STOP_REL 1e-10
#define PIVOT_REL 1e-12

typedef struct {
  double re, im;
} cplx;

/* Full-spectrum slot of harmonic k (in -kmax..kmax) and ring j. */
static int slot(int k, int j, int J, int kmax) { return (k + kmax) * J + j; }

/* Step 1: half spectrum (float or double) -> full Hermitian spectrum. */
static void expand_half_f(const float *h, int J, int kmax, cplx *F) {
  for (int k = 0; k <= kmax; ++k)
    for (int j = 0; j < J; ++j) {
      double re = h[(k * J + j) * 2 + 0];
      double im = (k == 0) ? 0.0 : h[(k * J + j) * 2 + 1];
      F[slot(k, j, J, kmax)].re = re;
      F[slot(k, j, J, kmax)].im = im;
      F[slot(-k, j, J, kmax)].re = re;
      F[slot(-k, j, J, kmax)].im = -im;
    }
}

static void expand_half_d(const double *h, int J, int kmax, cplx *F) {
  for (int k = 0; k <= kmax; ++k)
    for (int j = 0; j < J; ++j) {
      double re = h[(k * J + j) * 2 + 0];
      double im = (k == 0) ? 0.0 : h[(k * J + j) * 2 + 1];
      F[slot(k, j, J, kmax)].re = re;
      F[slot(k, j, J, kmax)].im = im;
      F[slot(-k, j, J, kmax)].re = re;
      F[slot(-k, j, J, kmax)].im = -im;
    }
}

/* Coefficient-space inner product of Eq. (rearrange): Re sum conj(u) v over
 * the full spectrum.  For Hermitian spectra the sum is real already. */
static double inner(const cplx *U, const cplx *V, int nq) {
  double s = 0.0;
  for (int q = 0; q < nq; ++q) s += U[q].re * V[q].re + U[q].im * V[q].im;
  return s;
}

/* Steering matrix of Eq. (Sr): harmonic k is multiplied by exp(-i k theta). */
static void steer(const cplx *F, int J, int kmax, double theta, cplx *out) {
  for (int k = -kmax; k <= kmax; ++k) {
    double c = cos(k * theta), s = -sin(k * theta);
    for (int j = 0; j < J; ++j) {
      cplx a = F[slot(k, j, J, kmax)];
      cplx *o = &out[slot(k, j, J, kmax)];
      o->re = c * a.re - s * a.im;
      o->im = c * a.im + s * a.re;
    }
  }
}

/* Step 2: the augmented dictionary [S_0 D ... S_{R-1} D], column m*R + r. */
static cplx *build_augmented(const float *d, int M, int J, int kmax, int R) {
  int nq = (2 * kmax + 1) * J;
  int hs = (kmax + 1) * J * 2;
  cplx *Fd = (cplx *)malloc(sizeof(cplx) * nq);
  cplx *A = (cplx *)malloc(sizeof(cplx) * (size_t)M * R * nq);
  if (!Fd || !A) {
    free(Fd);
    free(A);
    return NULL;
  }
  for (int m = 0; m < M; ++m) {
    expand_half_f(d + (size_t)m * hs, J, kmax, Fd);
    for (int r = 0; r < R; ++r)
      steer(Fd, J, kmax, 2.0 * M_PI * r / R, A + ((size_t)m * R + r) * nq);
  }
  free(Fd);
  return A;
}

/* Plain Cholesky of the t x t SPD matrix G (row-major) into L (lower).
 * Returns 0 if some pivot^2 <= PIVOT_REL * G_ii (degenerate support). */
static int cholesky(const double *G, int t, int ld, double *L) {
  for (int i = 0; i < t; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = G[i * ld + j];
      for (int k = 0; k < j; ++k) s -= L[i * ld + k] * L[j * ld + k];
      if (i == j) {
        if (!(s > PIVOT_REL * G[i * ld + i])) return 0;
        L[i * ld + i] = sqrt(s);
      } else {
        L[i * ld + j] = s / L[j * ld + j];
      }
    }
  }
  return 1;
}

/* Solve L L^T a = b. */
static void chol_solve(const double *L, int t, int ld, const double *b, double *a) {
  double z[64];
  for (int i = 0; i < t; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * ld + k] * z[k];
    z[i] = s / L[i * ld + i];
  }
  for (int i = t - 1; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < t; ++k) s -= L[k * ld + i] * a[k];
    a[i] = s / L[i * ld + i];
  }
}

/*
 * Step 3 for one patch.  forced_atom/forced_angle (length K) are NULL in free
 * mode; otherwise the picks are taken from them (forced-path mode, used to
 * check a different coder's picks and to give reference coefficients along
 * its path).  Outputs are length K except rn2.
 */
static void omp_patch(const float *xh, const cplx *Aug, int M, int R, int J, int kmax, int K,
                      const int32_t *forced_atom, const int32_t *forced_angle, int32_t *atom,
                      int32_t *angle, double *coef, double *rn2, double *margin, double *pick_s,
                      double *best_s, cplx *X, cplx *res) {
  int nq = (2 * kmax + 1) * J;
  int MR = M * R;
  int sel[64];
  double G[64 * 64], L[64 * 64], b[64], a[64];
  int t = 0;

  expand_half_f(xh, J, kmax, X);
  memcpy(res, X, sizeof(cplx) * nq);
  double xnorm = sqrt(inner(X, X, nq));

  for (int i = 0; i < K; ++i) {
    atom[i] = -1;
    angle[i] = -1;
    coef[i] = 0.0;
    if (margin) margin[i] = -1.0;
    if (pick_s) pick_s[i] = -1.0;
    if (best_s) best_s[i] = -1.0;
  }

  for (int step = 0; step < K; ++step) {
    /* scores of every steered atom against the residual */
    int best = -1;
    double s1 = -1.0, s2 = -1.0;
    for (int c = 0; c < MR; ++c) {
      double s = fabs(inner(Aug + (size_t)c * nq, res, nq));
      if (s > s1) {
        s2 = s1;
        s1 = s;
        best = c;
      } else if (s > s2) {
        s2 = s;
      }
    }
    if (s2 < 0.0) s2 = 0.0;
    if (best_s) best_s[step] = s1;
    if (margin) margin[step] = (s1 > 0.0) ? (s1 - s2) / s1 : 0.0;

    int pick = best;
    if (forced_atom) {
      if (forced_atom[step] < 0) break;
      pick = forced_atom[step] * R + forced_angle[step];
      if (pick_s) pick_s[step] = fabs(inner(Aug + (size_t)pick * nq, res, nq));
    } else if (!(s1 > STOP_REL * xnorm)) {
      break; /* nothing left to explain */
    }

    /* least squares over the enlarged support, Gram rebuilt from scratch */
    sel[t] = pick;
    int tt = t + 1;
    for (int p = 0; p < tt; ++p) {
      for (int q = 0; q < tt; ++q)
        G[p * 64 + q] = inner(Aug + (size_t)sel[p] * nq, Aug + (size_t)sel[q] * nq, nq);
      b[p] = inner(Aug + (size_t)sel[p] * nq, X, nq);
    }
    if (!cholesky(G, tt, 64, L)) break; /* degenerate: the new atom adds nothing */
    chol_solve(L, tt, 64, b, a);
    t = tt;

    memcpy(res, X, sizeof(cplx) * nq);
    for (int p = 0; p < t; ++p) {
      const cplx *Ap = Aug + (size_t)sel[p] * nq;
      for (int q = 0; q < nq; ++q) {
        res[q].re -= a[p] * Ap[q].re;
        res[q].im -= a[p] * Ap[q].im;
      }
    }
  }

  for (int p = 0; p < t; ++p) {
    atom[p] = sel[p] / R;
    angle[p] = sel[p] % R;
    coef[p] = a[p];
  }
  *rn2 = inner(res, res, nq);
}

/*
 * Rotational OMP over P patches.
 *   x      : P x (kmax+1) x J x 2 floats (half spectra)
 *   d      : M x (kmax+1) x J x 2 floats (unit-norm atoms)
 *   outputs: atom, angle (int32, P x K, -1 where no step), coef (P x K),
 *            rn2 (P, squared residual norm), margin (P x K or NULL:
 *            (s1 - s2) / s1 of the exact scores at each step).
 *   forced_atom / forced_angle: NULL (free mode) or P x K picks to follow.
 *   pick_s / best_s: NULL or P x K; |score| of the pick and the max |score|.
 * Returns 0 on success, -1 on bad arguments or allocation failure.
 */
int rsc_oracle_romp(const float *x, int64_t P, const float *d, int M, int J, int kmax, int R,
                    int K, const int32_t *forced_atom, const int32_t *forced_angle, int32_t *atom,
                    int32_t *angle, double *coef, double *rn2, double *margin, double *pick_s,
                    double *best_s, int nthreads) {
  if (P < 0 || M < 1 || J < 1 || kmax < 0 || R < 1 || K < 1 || K > 64) return -1;
  if (P == 0) return 0;
  cplx *Aug = build_augmented(d, M, J, kmax, R);
  if (!Aug) return -1;
  int nq = (2 * kmax + 1) * J;
  int hs = (kmax + 1) * J * 2;
  int failed = 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
  {
    cplx *X = (cplx *)malloc(sizeof(cplx) * nq);
    cplx *res = (cplx *)malloc(sizeof(cplx) * nq);
    if (!X || !res) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      failed = 1;
    } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
      for (int64_t p = 0; p < P; ++p) {
        omp_patch(x + p * hs, Aug, M, R, J, kmax, K, forced_atom ? forced_atom + p * K : NULL,
                  forced_angle ? forced_angle + p * K : NULL, atom + p * K, angle + p * K,
                  coef + p * K, rn2 + p, margin ? margin + p * K : NULL,
                  pick_s ? pick_s + p * K : NULL, best_s ? best_s + p * K : NULL, X, res);
      }
    }
    free(X);
    free(res);
  }
  free(Aug);
  (void)nthreads;
  return failed ? -1 : 0;
}

/* Exact scores <S_r d_m, x> for one patch, all m and r (flat index m*R + r).
 * Used by the pins; not part of the OMP loop above. */
int rsc_oracle_scores(const float *xh, const float *d, int M, int J, int kmax, int R,
                      double *scores) {
  int nq = (2 * kmax + 1) * J;
  cplx *Aug = build_augmented(d, M, J, kmax, R);
  cplx *X = (cplx *)malloc(sizeof(cplx) * nq);
  if (!Aug || !X) {
    free(Aug);
    free(X);
    return -1;
  }
  expand_half_f(xh, J, kmax, X);
  for (int c = 0; c < M * R; ++c) scores[c] = inner(Aug + (size_t)c * nq, X, nq);
  free(Aug);
  free(X);
  return 0;
}

/* Steer one FP64 half spectrum by an arbitrary angle theta (Eq. (Sr) with a
 * continuous angle); writes the half spectrum of the result. */
void rsc_oracle_steer(const double *in, int J, int kmax, double theta, double *out) {
  int nq = (2 * kmax + 1) * J;
  cplx *F = (cplx *)malloc(sizeof(cplx) * nq);
  cplx *G = (cplx *)malloc(sizeof(cplx) * nq);
  expand_half_d(in, J, kmax, F);
  steer(F, J, kmax, theta, G);
  for (int k = 0; k <= kmax; ++k)
    for (int j = 0; j < J; ++j) {
      out[(k * J + j) * 2 + 0] = G[slot(k, j, J, kmax)].re;
      out[(k * J + j) * 2 + 1] = (k == 0) ? 0.0 : G[slot(k, j, J, kmax)].im;
    }
  free(F);
  free(G);
}

/* Coefficient-space inner product of two FP64 half spectra (via the full
 * Hermitian spectrum). */
double rsc_oracle_inner(const double *u, const double *v, int J, int kmax) {
  int nq = (2 * kmax + 1) * J;
  cplx *U = (cplx *)malloc(sizeof(cplx) * nq);
  cplx *V = (cplx *)malloc(sizeof(cplx) * nq);
  expand_half_d(u, J, kmax, U);
  expand_half_d(v, J, kmax, V);
  double s = inner(U, V, nq);
  free(U);
  free(V);
  return s;
}

int rsc_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
