/*
 * CPU oracle for the symmetry-preserving random batch Ewald (SRBE) method for
 * constant-potential electrode/electrolyte slabs (Gao, Zhou, Zhang, Xu,
 * arXiv 2509.24742).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the CPU-baseline leg of the benchmark call it; the library never does.
 *
 * Plain FP64 loops that follow the paper's formulas term by term.  Units are
 * "Gaussian" (energy = q q' / r, potential = q / r); the Python side multiplies
 * energies and forces by the Coulomb constant.  Arrays of vectors are row-major
 * [n][3].  Equation numbers count the displayed equations of the paper in order
 * (Eq. 18 = the matrix A, Eq. 19 = the vector b, Eq. 24 = SRBE b, Eq. 25 = SRBE
 * force, Eqs. 26-29 = the sampling law and the Metropolis step).
 *
 * Readings where the paper is garbled or silent (each pinned by a test):
 *  - the slab term of A is (4 pi / V) Z_i Z_j, the Hessian of (2 pi / V) M_z^2;
 *  - the slab term of b is -(4 pi Z_j / V) sum_i q_i z_i, so b = -dU/dQ at Q = 0;
 *  - b carries no "+ delta psi"; the voltage enters only through delta psi * d;
 *  - eta is the Gaussian width as a length (exp(-r^2 / eta^2), Eq. 1).
 * Parity of every function here is pinned by the not-gpu tests in tests/.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------------
 * Neumaier-compensated summation (order-independent to about 1 ulp of the sum)
 * ------------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;

static void nadd(nsum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* ---------------------------------------------------------------------------
 * Fourier modes: k = 2 pi m / L (componentwise), Eq. 16 (the lattice L_k)
 * ------------------------------------------------------------------------- */
void orc_kvectors(const double L[3], int64_t K, const int32_t *m, double *kv) {
  for (int64_t k = 0; k < K; ++k)
    for (int d = 0; d < 3; ++d) kv[3 * k + d] = 2.0 * M_PI * (double)m[3 * k + d] / L[d];
}

/* Structure factor S(k) = sum_j q_j exp(i k . r_j), Eq. 15; S is [K][2] (re, im). */
void orc_sfac(int64_t n, const double *r, const double *q, int64_t K, const double *kv, double *S) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < K; ++k) {
    nsum re = {0, 0}, im = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      double ph = kv[3 * k] * r[3 * j] + kv[3 * k + 1] * r[3 * j + 1] + kv[3 * k + 2] * r[3 * j + 2];
      nadd(&re, q[j] * cos(ph));
      nadd(&im, q[j] * sin(ph));
    }
    S[2 * k] = nval(&re);
    S[2 * k + 1] = nval(&im);
  }
}

/* Far-field part of b for a weighted mode list:
 *   b_F,j = - sum_k c_k Re( exp(-i k . R_j) S1(k) ),
 * with c_k = 4 pi exp(-k^2 / 4 alpha^2) / (V k^2) for every mode of L_k (Eq. 20)
 * or for the deterministic set I, and c_k = (G / P) 4 pi / (V k^2) for each
 * sampled mode (Eq. 24). */
void orc_b_far(int64_t ne, const double *R, int64_t K, const double *kv, const double *c,
               const double *S1, double *bF) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < ne; ++j) {
    nsum acc = {0, 0};
    for (int64_t k = 0; k < K; ++k) {
      double ph = kv[3 * k] * R[3 * j] + kv[3 * k + 1] * R[3 * j + 1] + kv[3 * k + 2] * R[3 * j + 2];
      /* Re(exp(-i ph) (Sr + i Si)) = cos(ph) Sr + sin(ph) Si */
      nadd(&acc, -c[k] * (cos(ph) * S1[2 * k] + sin(ph) * S1[2 * k + 1]));
    }
    bF[j] = nval(&acc);
  }
}

/* Ion-electrode real-space kernel of Eq. 13: [erfc(alpha d) - erfc(d / eta)] / d. */
static double phi_ie(double d, double alpha, double eta) {
  return (erfc(alpha * d) - erfc(d / eta)) / d;
}
/* Electrode-electrode real-space kernel of Eq. 13 / Eq. 18. */
static double phi_ee(double d, double alpha, double eta) {
  return (erfc(alpha * d) - erfc(d / (sqrt(2.0) * eta))) / d;
}

/* Number of in-plane periodic images to scan so that every image within rc of
 * a wrapped displacement is visited (rc may exceed half the box). */
static int n_images(double rc, double L) { return (int)ceil(rc / L) + 1; }

/* Near-field part of b, third term of Eq. 19:
 *   b_N,j = - sum_i sum_{n in Z^2 x {0}} q_i phi_ie(|R_j - r_i - n o l|), |.| < rc. */
void orc_b_near(const double L[3], double alpha, double eta, double rc, int64_t ni, const double *r,
                const double *q, int64_t ne, const double *R, double *bN) {
  int nx = n_images(rc, L[0]), ny = n_images(rc, L[1]);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < ne; ++j) {
    nsum acc = {0, 0};
    for (int64_t i = 0; i < ni; ++i) {
      double dx0 = R[3 * j] - r[3 * i], dy0 = R[3 * j + 1] - r[3 * i + 1], dz = R[3 * j + 2] - r[3 * i + 2];
      dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
      dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
      for (int a = -nx; a <= nx; ++a)
        for (int b = -ny; b <= ny; ++b) {
          double dx = dx0 + a * L[0], dy = dy0 + b * L[1];
          double d = sqrt(dx * dx + dy * dy + dz * dz);
          if (d < rc) nadd(&acc, -q[i] * phi_ie(d, alpha, eta));
        }
    }
    bN[j] = nval(&acc);
  }
}

/* Slab-correction part of b (reading of Eq. 19, pinned by finite differences):
 *   b_slab,j = -(4 pi / V) Z_j sum_i q_i z_i. */
void orc_b_slab(const double L[3], int64_t ni, const double *r, const double *q, int64_t ne,
                const double *R, double *bS) {
  double V = L[0] * L[1] * L[2];
  nsum m = {0, 0};
  for (int64_t i = 0; i < ni; ++i) nadd(&m, q[i] * r[3 * i + 2]);
  double Mi = nval(&m);
  for (int64_t j = 0; j < ne; ++j) bS[j] = -(4.0 * M_PI / V) * R[3 * j + 2] * Mi;
}

/* Matrix A of Eq. 18 (slab term read as (4 pi / V) Z_i Z_j), for a given mode
 * list (every nonzero k of the truncated lattice) and real-space cutoff:
 *   A_ij = (1/V) sum_k 4 pi / k^2 exp(-k^2/4a^2) cos(k . (R_i - R_j))
 *        + sum'_{n} phi_ee(|R_i - R_j + n o l|)
 *        + 2 delta_ij (1 / (sqrt(2 pi) eta) - a / sqrt(pi)) + (4 pi / V) Z_i Z_j.
 * cos(k.(R_i - R_j)) is expanded as cos_i cos_j + sin_i sin_j. */
void orc_build_A(const double L[3], double alpha, double eta, double rcut, int64_t K, const int32_t *m,
                 int64_t ne, const double *R, double *A) {
  double V = L[0] * L[1] * L[2];
  double *kv = (double *)malloc(sizeof(double) * 3 * (K > 0 ? K : 1));
  double *w = (double *)malloc(sizeof(double) * (K > 0 ? K : 1));
  double *cs = (double *)malloc(sizeof(double) * 2 * (K > 0 ? K : 1) * ne);
  orc_kvectors(L, K, m, kv);
  for (int64_t k = 0; k < K; ++k) {
    double k2 = kv[3 * k] * kv[3 * k] + kv[3 * k + 1] * kv[3 * k + 1] + kv[3 * k + 2] * kv[3 * k + 2];
    w[k] = 4.0 * M_PI / (V * k2) * exp(-k2 / (4.0 * alpha * alpha));
  }
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < ne; ++j)
    for (int64_t k = 0; k < K; ++k) {
      double ph = kv[3 * k] * R[3 * j] + kv[3 * k + 1] * R[3 * j + 1] + kv[3 * k + 2] * R[3 * j + 2];
      cs[2 * (j * K + k)] = cos(ph);
      cs[2 * (j * K + k) + 1] = sin(ph);
    }
  int nx = n_images(rcut, L[0]), ny = n_images(rcut, L[1]);
  double self = 2.0 * (1.0 / (sqrt(2.0 * M_PI) * eta) - alpha / sqrt(M_PI));
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < ne; ++i) {
    for (int64_t j = i; j < ne; ++j) {
      nsum acc = {0, 0};
      const double *ci = cs + 2 * i * K, *cj = cs + 2 * j * K;
      for (int64_t k = 0; k < K; ++k) nadd(&acc, w[k] * (ci[2 * k] * cj[2 * k] + ci[2 * k + 1] * cj[2 * k + 1]));
      double dx0 = R[3 * i] - R[3 * j], dy0 = R[3 * i + 1] - R[3 * j + 1], dz = R[3 * i + 2] - R[3 * j + 2];
      dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
      dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
      for (int a = -nx; a <= nx; ++a)
        for (int b = -ny; b <= ny; ++b) {
          double dx = dx0 + a * L[0], dy = dy0 + b * L[1];
          double d = sqrt(dx * dx + dy * dy + dz * dz);
          if (d > 0.0 && d < rcut) nadd(&acc, phi_ee(d, alpha, eta));
        }
      if (i == j) nadd(&acc, self);
      nadd(&acc, 4.0 * M_PI / V * R[3 * i + 2] * R[3 * j + 2]);
      A[i * ne + j] = A[j * ne + i] = nval(&acc);
    }
  }
  free(kv); free(w); free(cs);
}

/* Far-field force on ion i for a weighted mode list (Eq. 21 with all modes,
 * Eq. 25 with the SRBE list):
 *   F_i = - q_i sum_k c_k k Im( S(k) exp(-i k . r_i) ),  S = S1 + S2. */
void orc_force_kspace(int64_t ni, const double *r, const double *q, int64_t K, const double *kv,
                      const double *c, const double *S, double *F) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < ni; ++i) {
    nsum f[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t k = 0; k < K; ++k) {
      double ph = kv[3 * k] * r[3 * i] + kv[3 * k + 1] * r[3 * i + 1] + kv[3 * k + 2] * r[3 * i + 2];
      /* Im((Sr + i Si)(cos ph - i sin ph)) = Si cos ph - Sr sin ph */
      double im = S[2 * k + 1] * cos(ph) - S[2 * k] * sin(ph);
      for (int d = 0; d < 3; ++d) nadd(&f[d], -q[i] * c[k] * kv[3 * k + d] * im);
    }
    for (int d = 0; d < 3; ++d) F[3 * i + d] = nval(&f[d]);
  }
}

/* Slab (k = 0) force, the gradient of +(2 pi / V) M_z^2 (Eq. 17 enters U with a minus sign):
 *   F_i,z = -(4 pi / V) q_i M_z,  M_z = sum q_i z_i + sum Q_j Z_j. */
double orc_dipole_z(int64_t ni, const double *r, const double *q, int64_t ne, const double *R, const double *Q) {
  nsum m = {0, 0};
  for (int64_t i = 0; i < ni; ++i) nadd(&m, q[i] * r[3 * i + 2]);
  for (int64_t j = 0; j < ne; ++j) nadd(&m, Q[j] * R[3 * j + 2]);
  return nval(&m);
}

/* Real-space Coulomb forces and energies of Eq. 13 (ion-ion and ion-electrode
 * terms) for all images within rc.  E[0] = ion-ion, E[1] = ion-electrode.
 * F_i = - dU/dr_i; for a pair kernel phi(d):  F_i = - q_i q_j phi'(d) (r_i - r_j)/d.
 * With targets != NULL only the nt ions targets[0..nt) are evaluated (row t of F is
 * ion targets[t]; E then sums over those ions only); with NULL, nt is ignored and
 * every ion is a target. */
void orc_force_real(const double L[3], double alpha, double eta, double rc, int64_t ni, const double *r,
                    const double *q, int64_t ne, const double *R, const double *Q, int64_t nt,
                    const int64_t *targets, double *F, double *E) {
  int nx = n_images(rc, L[0]), ny = n_images(rc, L[1]);
  const double tpa = 2.0 / sqrt(M_PI);
  double eii = 0.0, eie = 0.0;
  if (!targets) nt = ni;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : eii, eie)
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t i = targets ? targets[t] : t;
    nsum f[3] = {{0, 0}, {0, 0}, {0, 0}};
    nsum ui = {0, 0}, ue = {0, 0};
    for (int64_t j = 0; j < ni; ++j) {
      double dx0 = r[3 * i] - r[3 * j], dy0 = r[3 * i + 1] - r[3 * j + 1], dz = r[3 * i + 2] - r[3 * j + 2];
      dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
      dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
      for (int a = -nx; a <= nx; ++a)
        for (int b = -ny; b <= ny; ++b) {
          if (j == i && a == 0 && b == 0) continue;
          double dx = dx0 + a * L[0], dy = dy0 + b * L[1];
          double d2 = dx * dx + dy * dy + dz * dz, d = sqrt(d2);
          if (d >= rc) continue;
          /* phi = erfc(a d)/d ; -phi' = erfc(a d)/d^2 + (2a/sqrt(pi)) exp(-a^2 d^2)/d */
          double mdphi = erfc(alpha * d) / d2 + tpa * alpha * exp(-alpha * alpha * d2) / d;
          double s = q[i] * q[j] * mdphi / d;
          nadd(&f[0], s * dx); nadd(&f[1], s * dy); nadd(&f[2], s * dz);
          nadd(&ui, 0.5 * q[i] * q[j] * erfc(alpha * d) / d);
        }
    }
    for (int64_t j = 0; j < ne; ++j) {
      double dx0 = r[3 * i] - R[3 * j], dy0 = r[3 * i + 1] - R[3 * j + 1], dz = r[3 * i + 2] - R[3 * j + 2];
      dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
      dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
      for (int a = -nx; a <= nx; ++a)
        for (int b = -ny; b <= ny; ++b) {
          double dx = dx0 + a * L[0], dy = dy0 + b * L[1];
          double d2 = dx * dx + dy * dy + dz * dz, d = sqrt(d2);
          if (d >= rc) continue;
          /* phi_ie = [erfc(a d) - erfc(d/eta)]/d */
          double mdphi = erfc(alpha * d) / d2 + tpa * alpha * exp(-alpha * alpha * d2) / d
                       - erfc(d / eta) / d2 - tpa / eta * exp(-d2 / (eta * eta)) / d;
          double s = q[i] * Q[j] * mdphi / d;
          nadd(&f[0], s * dx); nadd(&f[1], s * dy); nadd(&f[2], s * dz);
          nadd(&ue, q[i] * Q[j] * phi_ie(d, alpha, eta));
        }
    }
    for (int d = 0; d < 3; ++d) F[3 * t + d] = nval(&f[d]);
    eii += nval(&ui);
    eie += nval(&ue);
  }
  E[0] = eii;
  E[1] = eie;
}

/* Electrode-electrode real-space energy of Eq. 13 (third term) within rc. */
double orc_energy_ee_real(const double L[3], double alpha, double eta, double rc, int64_t ne, const double *R,
                          const double *Q) {
  int nx = n_images(rc, L[0]), ny = n_images(rc, L[1]);
  double e = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : e)
  for (int64_t i = 0; i < ne; ++i) {
    nsum u = {0, 0};
    for (int64_t j = 0; j < ne; ++j) {
      double dx0 = R[3 * i] - R[3 * j], dy0 = R[3 * i + 1] - R[3 * j + 1], dz = R[3 * i + 2] - R[3 * j + 2];
      dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
      dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
      for (int a = -nx; a <= nx; ++a)
        for (int b = -ny; b <= ny; ++b) {
          double dx = dx0 + a * L[0], dy = dy0 + b * L[1];
          double d = sqrt(dx * dx + dy * dy + dz * dz);
          if (d > 0.0 && d < rc) nadd(&u, 0.5 * Q[i] * Q[j] * phi_ee(d, alpha, eta));
        }
    }
    e += nval(&u);
  }
  return e;
}

/* Lennard-Jones 12-6 (plain truncation at rc, no shift) between ion sites of
 * different molecules and between ions and electrode sites, and harmonic bonds.
 * These are the MD support terms of the coarse-grained electrolyte (§4); they
 * are in kJ/mol already.  sig/eps are ntype x ntype tables; electrode type = etype. */
double orc_force_lj(const double L[3], double rc, int64_t ni, const double *r, const int32_t *mol,
                    const int32_t *typ, int64_t ne, const double *R, int32_t etype, int32_t ntype,
                    const double *sig, const double *eps, double *F) {
  int nx = n_images(rc, L[0]), ny = n_images(rc, L[1]);
  double etot = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : etot)
  for (int64_t i = 0; i < ni; ++i) {
    nsum f[3] = {{0, 0}, {0, 0}, {0, 0}}, u = {0, 0};
    for (int64_t j = 0; j < ni + ne; ++j) {
      int ion = j < ni;
      if (ion && mol[j] == mol[i]) continue;
      const double *p = ion ? r + 3 * j : R + 3 * (j - ni);
      int tj = ion ? typ[j] : etype;
      double s = sig[typ[i] * ntype + tj], e = eps[typ[i] * ntype + tj];
      double dx0 = r[3 * i] - p[0], dy0 = r[3 * i + 1] - p[1], dz = r[3 * i + 2] - p[2];
      dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
      dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
      for (int a = -nx; a <= nx; ++a)
        for (int b = -ny; b <= ny; ++b) {
          double dx = dx0 + a * L[0], dy = dy0 + b * L[1];
          double d2 = dx * dx + dy * dy + dz * dz;
          if (d2 >= rc * rc) continue;
          double sr2 = s * s / d2, sr6 = sr2 * sr2 * sr2;
          /* U = 4 e (sr12 - sr6); F = 24 e (2 sr12 - sr6) / d^2 * dvec */
          double fs = 24.0 * e * (2.0 * sr6 * sr6 - sr6) / d2;
          nadd(&f[0], fs * dx); nadd(&f[1], fs * dy); nadd(&f[2], fs * dz);
          nadd(&u, (ion ? 0.5 : 1.0) * 4.0 * e * (sr6 * sr6 - sr6));
        }
    }
    for (int d = 0; d < 3; ++d) F[3 * i + d] = nval(&f[d]);
    etot += nval(&u);
  }
  return etot;
}

double orc_force_bonds(const double L[3], int64_t nb, const int32_t *bonds, const double *r0, double kb,
                       const double *r, double *F) {
  double e = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    int64_t i = bonds[2 * b], j = bonds[2 * b + 1];
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = r[3 * i + a] - r[3 * j + a];
    d[0] -= L[0] * floor(d[0] / L[0] + 0.5);
    d[1] -= L[1] * floor(d[1] / L[1] + 0.5);
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double f = -kb * (len - r0[b]) / len;  /* U = kb/2 (len - r0)^2 */
    for (int a = 0; a < 3; ++a) { F[3 * i + a] += f * d[a]; F[3 * j + a] -= f * d[a]; }
    e += 0.5 * kb * (len - r0[b]) * (len - r0[b]);
  }
  return e;
}

/* ---------------------------------------------------------------------------
 * Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): a counter-based generator
 * with multipliers 0xD2E7470EE14C6C93, 0xCA5A826395121157 and Weyl key
 * increments 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B.
 * ------------------------------------------------------------------------- */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B97F4A7C15ull; k1 += 0xBB67AE8584CAA73Bull; }
    uint64_t h0, l0, h1, l1;
    mulhilo64(0xD2E7470EE14C6C93ull, c0, &h0, &l0);
    mulhilo64(0xCA5A826395121157ull, c2, &h1, &l1);
    uint64_t n0 = h1 ^ c1 ^ k0, n1 = l1, n2 = h0 ^ c3 ^ k1, n3 = l0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform on (0, 1] from the top 53 bits */
static double u01(uint64_t x) { return ((double)(x >> 11) + 1.0) * 0x1.0p-53; }

/* Random draws for proposal j of step `step`: three standard normals (Box-Muller
 * on the first four words) and one uniform for the acceptance test.  Key =
 * (seed, 0x5352424500000001), counters (2j, step, 0, 0) and (2j + 1, step, 0, 0). */
static void draws(uint64_t seed, uint64_t step, uint64_t j, double nrm[3], double *uacc) {
  uint64_t key[2] = {seed, 0x5352424500000001ull};
  uint64_t c0[4] = {2 * j, step, 0, 0}, c1[4] = {2 * j + 1, step, 0, 0}, o0[4], o1[4];
  orc_philox4x64(c0, key, o0);
  orc_philox4x64(c1, key, o1);
  double r1 = sqrt(-2.0 * log(u01(o0[0]))), t1 = 2.0 * M_PI * u01(o0[1]);
  double r2 = sqrt(-2.0 * log(u01(o0[2]))), t2 = 2.0 * M_PI * u01(o0[3]);
  nrm[0] = r1 * cos(t1);
  nrm[1] = r1 * sin(t1);
  nrm[2] = r2 * cos(t2);
  *uacc = u01(o1[0]);
}

/* Per-dimension width of the target: exp(-k_d^2 / 4 a^2) = exp(-pi^2 m^2 / (a L_d)^2),
 * a discrete Gaussian with sigma_d = a L_d / (sqrt(2) pi) (reading of Eqs. 26, 28). */
static double sigma_d(double alpha, double Ld) { return alpha * Ld / (sqrt(2.0) * M_PI); }

/* The excluded set: k = 0 and the deterministic modes I = {(0, 0, m_z): 1 <= |m_z| <= M}
 * (after Eq. 25), plus anything outside an optional truncation box |m_d| <= mmax_d
 * (mmax_d <= 0 means no box). */
static int excluded(const int32_t m[3], int M, const int32_t mmax[3]) {
  for (int d = 0; d < 3; ++d)
    if (mmax[d] > 0 && abs(m[d]) > mmax[d]) return 1;
  return m[0] == 0 && m[1] == 0 && abs(m[2]) <= M;
}

/* q_d(m) of Eq. 28: the mass of N(0, sigma_d^2) on [m - 1/2, m + 1/2]. */
static double qd(int32_t m, double sig) {
  double s = sqrt(2.0) * sig;
  return 0.5 * (erf((m + 0.5) / s) - erf((m - 0.5) / s));
}

/* exp(-k^2 / 4 alpha^2) for integer m, the unnormalised P(k) of Eq. 26. */
static double pk(const int32_t m[3], const double L[3], double alpha) {
  double k2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    double kd = 2.0 * M_PI * m[d] / L[d];
    k2 += kd * kd;
  }
  return exp(-k2 / (4.0 * alpha * alpha));
}

/* Metropolis sampling of P modes from P(k) on L_k \ I (Eqs. 26-29).  Proposals
 * are independent rounded Gaussians per dimension (round = floor(x + 1/2));
 * the chain starts at the first proposal outside I u {0} (the step has no
 * earlier state), proposals inside I u {0} (or outside the box) are rejected,
 * and the P consecutive chain states are returned.  Returns the number of
 * proposals used. */
int64_t orc_sample_metropolis(const double L[3], double alpha, int M, const int32_t mmax[3], int P,
                              uint64_t seed, uint64_t step, int32_t *m_out) {
  double sig[3];
  for (int d = 0; d < 3; ++d) sig[d] = sigma_d(alpha, L[d]);
  uint64_t j = 0;
  int32_t cur[3];
  double nrm[3], u;
  for (;;) { /* initial state */
    draws(seed, step, j++, nrm, &u);
    for (int d = 0; d < 3; ++d) cur[d] = (int32_t)floor(sig[d] * nrm[d] + 0.5);
    if (!excluded(cur, M, mmax)) break;
  }
  double pcur = pk(cur, L, alpha), qcur = qd(cur[0], sig[0]) * qd(cur[1], sig[1]) * qd(cur[2], sig[2]);
  for (int l = 0; l < P; ++l) {
    if (l > 0) {
      int32_t prop[3];
      draws(seed, step, j++, nrm, &u);
      for (int d = 0; d < 3; ++d) prop[d] = (int32_t)floor(sig[d] * nrm[d] + 0.5);
      if (!excluded(prop, M, mmax)) {
        double pp = pk(prop, L, alpha);
        double qp = qd(prop[0], sig[0]) * qd(prop[1], sig[1]) * qd(prop[2], sig[2]);
        /* a = min{1, P(k*) q(m) / (P(k) q(m*))}, Eq. 29 (G cancels) */
        double a = (pp * qcur) / (pcur * qp);
        if (u <= a) {
          for (int d = 0; d < 3; ++d) cur[d] = prop[d];
          pcur = pp;
          qcur = qp;
        }
      }
    }
    for (int d = 0; d < 3; ++d) m_out[3 * l + d] = cur[d];
  }
  return (int64_t)j;
}

/* Support bound used when no box is given: exp(-pi^2 m^2 / (a L)^2) < 1e-21. */
static int32_t support(double alpha, double Ld, int32_t mmax) {
  if (mmax > 0) return mmax;
  return (int32_t)ceil(alpha * Ld * sqrt(21.0 * log(10.0)) / M_PI);
}

/* Exact i.i.d. sampler of P(k) on L_k \ I: inverse-CDF draw of each dimension's
 * discrete Gaussian (P(k) is a product over dimensions), rejecting I u {0}. */
int64_t orc_sample_exact(const double L[3], double alpha, int M, const int32_t mmax[3], int P, uint64_t seed,
                         uint64_t step, int32_t *m_out) {
  int32_t sup[3];
  double *cdf[3];
  for (int d = 0; d < 3; ++d) {
    sup[d] = support(alpha, L[d], mmax[d]);
    int n = 2 * sup[d] + 1;
    cdf[d] = (double *)malloc(sizeof(double) * n);
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      double kd = 2.0 * M_PI * (i - sup[d]) / L[d];
      acc += exp(-kd * kd / (4.0 * alpha * alpha));
      cdf[d][i] = acc;
    }
    for (int i = 0; i < n; ++i) cdf[d][i] /= acc;
  }
  uint64_t key[2] = {seed, 0x5352424500000002ull};
  int64_t tries = 0;
  for (int l = 0; l < P;) {
    uint64_t ctr[4] = {(uint64_t)tries++, step, 1, 0}, o[4];
    orc_philox4x64(ctr, key, o);
    int32_t m[3];
    for (int d = 0; d < 3; ++d) {
      double u = u01(o[d]);
      int n = 2 * sup[d] + 1, i = 0;
      while (i < n - 1 && cdf[d][i] < u) ++i;
      m[d] = i - sup[d];
    }
    if (excluded(m, M, mmax)) continue;
    for (int d = 0; d < 3; ++d) m_out[3 * l + d] = m[d];
    ++l;
  }
  for (int d = 0; d < 3; ++d) free(cdf[d]);
  return tries;
}

/* G of Eq. 27 by direct summation over the (possibly truncated) lattice. */
double orc_G_brute(const double L[3], double alpha, int M, const int32_t mmax[3]) {
  int32_t s[3];
  for (int d = 0; d < 3; ++d) s[d] = support(alpha, L[d], mmax[d]);
  nsum g = {0, 0};
  for (int32_t a = -s[0]; a <= s[0]; ++a)
    for (int32_t b = -s[1]; b <= s[1]; ++b)
      for (int32_t c = -s[2]; c <= s[2]; ++c) {
        int32_t m[3] = {a, b, c};
        if (excluded(m, M, mmax)) continue;
        nadd(&g, pk(m, L, alpha));
      }
  return nval(&g);
}

/* Rows of A x (Eq. 18) without forming A: out[r] = sum_j A[rows[r]][j] x_j with the terms of
 * orc_build_A (full-lattice modes m [K][3], Gaussian-screened real-space images within rcut, self
 * term, slab term), the k-space part as sum_k w_k Re(exp(-i k.R_i) S_x(k)), S_x(k) = sum_j x_j
 * exp(i k.R_j).  For checks of a solve at sizes where A cannot be formed. */
void orc_A_rows(const double L[3], double alpha, double eta, double rcut, int64_t K, const int32_t *m, int64_t ne,
                const double *R, const double *x, int64_t nrow, const int64_t *rows, double *out) {
  double V = L[0] * L[1] * L[2];
  double *kv = (double *)malloc(sizeof(double) * 3 * (K > 0 ? K : 1));
  double *S = (double *)malloc(sizeof(double) * 2 * (K > 0 ? K : 1));
  orc_kvectors(L, K, m, kv);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < K; ++k) {
    nsum re = {0, 0}, im = {0, 0};
    for (int64_t j = 0; j < ne; ++j) {
      double ph = kv[3 * k] * R[3 * j] + kv[3 * k + 1] * R[3 * j + 1] + kv[3 * k + 2] * R[3 * j + 2];
      nadd(&re, x[j] * cos(ph));
      nadd(&im, x[j] * sin(ph));
    }
    S[2 * k] = nval(&re);
    S[2 * k + 1] = nval(&im);
  }
  int nx = n_images(rcut, L[0]), ny = n_images(rcut, L[1]);
  double self = 2.0 * (1.0 / (sqrt(2.0 * M_PI) * eta) - alpha / sqrt(M_PI));
  nsum mz = {0, 0};
  for (int64_t j = 0; j < ne; ++j) nadd(&mz, R[3 * j + 2] * x[j]);
  double Mz = nval(&mz);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrow; ++r) {
    int64_t i = rows[r];
    nsum acc = {0, 0};
    for (int64_t k = 0; k < K; ++k) {
      double k2 = kv[3 * k] * kv[3 * k] + kv[3 * k + 1] * kv[3 * k + 1] + kv[3 * k + 2] * kv[3 * k + 2];
      double w = 4.0 * M_PI / (V * k2) * exp(-k2 / (4.0 * alpha * alpha));
      double ph = kv[3 * k] * R[3 * i] + kv[3 * k + 1] * R[3 * i + 1] + kv[3 * k + 2] * R[3 * i + 2];
      /* Re((cos ph - i sin ph)(S_re + i S_im)) */
      nadd(&acc, w * (cos(ph) * S[2 * k] + sin(ph) * S[2 * k + 1]));
    }
    for (int64_t j = 0; j < ne; ++j) {
      double dx0 = R[3 * i] - R[3 * j], dy0 = R[3 * i + 1] - R[3 * j + 1], dz = R[3 * i + 2] - R[3 * j + 2];
      dx0 -= L[0] * floor(dx0 / L[0] + 0.5);
      dy0 -= L[1] * floor(dy0 / L[1] + 0.5);
      for (int a = -nx; a <= nx; ++a)
        for (int b = -ny; b <= ny; ++b) {
          double dx = dx0 + a * L[0], dy = dy0 + b * L[1];
          double d = sqrt(dx * dx + dy * dy + dz * dz);
          if (d > 0.0 && d < rcut) nadd(&acc, phi_ee(d, alpha, eta) * x[j]);
        }
    }
    nadd(&acc, self * x[i]);
    nadd(&acc, 4.0 * M_PI / V * R[3 * i + 2] * Mz);
    out[r] = nval(&acc);
  }
  free(kv); free(S);
}

/* ---------------------------------------------------------------------------
 * Langevin thermostat noise (Eq. 39: the Wiener increments dW_i of every ion).
 * Three independent standard normal numbers per ion i and step n: Philox4x64-10
 * with key (seed, 0x4C414E47) and counter (n, i, 0, 0) gives four 64-bit words
 * w0..w3; uniforms u_a = ((w_a >> 11) + 1/2) 2^-53 lie strictly inside (0, 1);
 * Box-Muller: g_x = sqrt(-2 ln u0) cos(2 pi u1), g_y = sqrt(-2 ln u0) sin(2 pi u1),
 * g_z = sqrt(-2 ln u2) cos(2 pi u3).  g is [n][3].
 * ------------------------------------------------------------------------- */
void orc_langevin_gauss(uint64_t seed, uint64_t step, int64_t n, double *g) {
  const uint64_t key[2] = {seed, 0x4C414E47ull};
  for (int64_t i = 0; i < n; ++i) {
    uint64_t ctr[4] = {step, (uint64_t)i, 0, 0}, w[4];
    orc_philox4x64(ctr, key, w);
    double u[4];
    for (int a = 0; a < 4; ++a) u[a] = ((double)(w[a] >> 11) + 0.5) * 0x1.0p-53;
    const double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    g[3 * i + 0] = r0 * cos(2.0 * M_PI * u[1]);
    g[3 * i + 1] = r0 * sin(2.0 * M_PI * u[1]);
    g[3 * i + 2] = r1 * cos(2.0 * M_PI * u[3]);
  }
}
