/*
 * Direct-sum oracle (no FFT) for the discrete operators of the paper.
 * TEST INFRASTRUCTURE ONLY: called from tests through ctypes (oracle/direct.py).
 *
 * Every array is n^3 doubles in cyclic order: flat index (c1*n + c2)*n + c3,
 * c_d = l_d mod n for the paper's multi-index l_d in {-N_p .. N_p-1}.
 *
 *  lbo_direct_linearized  -- Algorithm 1 of the paper (Eqs. (3.4)-(3.9)) written
 *     as real-space cyclic double convolutions, O(J n^6):
 *       r      = f / M  (0 where M/rho < eps, Eq. (3.9))
 *       psi_j  = (M^g phit_j) (*) r               (Eq. (3.8), divided by 8 pi^3)
 *       L+     = sum_j 4 pi^2 w_j B_j  phit_j (*) (M^h psi_j)     (Eq. (3.7))
 *       L-     = M (Omega (*) f) + f (Omega (*) M)                (Eq. (3.4))
 *     with phit_j = IDFT(s_j), Omega = IDFT(omega) evaluated as direct cosine
 *     sums (the multipliers are real and even).
 *
 *  lbo_direct_quadratic -- Eq. (2.14) with the convolution I_{j,k,m} summed
 *     directly in Fourier space, O(J M n^6); symmetric bilinear form
 *     Q(f,g)+Q(g,f) when g != NULL.  The Nyquist reading of the non-even
 *     multipliers is the same as in oracle/quadratic.py.
 *
 * The working precision is `real`: double here; direct_ld.c compiles this
 * file again with long double (extended precision, binary128 where the
 * platform's long double is) and the suffix _ld, as the reference for
 * inputs whose FP64 evaluations differ by u max|r|.  Inputs, tables and
 * outputs stay double; the cut-off decision of Eq. (3.9) is taken in
 * double, every operation rounded separately (build with -ffp-contract=off).
 */
#ifndef REAL
#define REAL double
#endif
#ifndef SUFFIX
#define SUFFIX(name) name
#endif
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

typedef REAL real;
#define PI_R ((real)3.14159265358979323846264338327950288L)

static int cen(int c, int n) { return c < n / 2 ? c : c - n; }
static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }
static real sincd(real x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* out[p] = n^{-3} sum_k mult[k] cos(2 pi k.p / n), mult real and even. */
static void idft_even(int n, const real *mult, real *out) {
  const int n3 = n * n * n;
  real *ct = (real *)malloc(sizeof(real) * n);
  for (int t = 0; t < n; ++t) ct[t] = cos(2.0 * PI_R * t / n);
  for (int p1 = 0; p1 < n; ++p1)
    for (int p2 = 0; p2 < n; ++p2)
      for (int p3 = 0; p3 < n; ++p3) {
        real acc = 0.0;
        for (int k1 = 0; k1 < n; ++k1)
          for (int k2 = 0; k2 < n; ++k2)
            for (int k3 = 0; k3 < n; ++k3) {
              int t = (k1 * p1 + k2 * p2 + k3 * p3) % n;
              acc += mult[(k1 * n + k2) * n + k3] * ct[t];
            }
        out[(p1 * n + p2) * n + p3] = acc / n3;
      }
  free(ct);
}

/* y[l] = sum_p a[p] b[l - p]  (cyclic) */
static void cyc_conv(int n, const real *a, const real *b, real *y) {
  for (int l1 = 0; l1 < n; ++l1)
    for (int l2 = 0; l2 < n; ++l2)
      for (int l3 = 0; l3 < n; ++l3) {
        real acc = 0.0;
        for (int p1 = 0; p1 < n; ++p1) {
          int q1 = wrap(l1 - p1, n);
          for (int p2 = 0; p2 < n; ++p2) {
            int q2 = wrap(l2 - p2, n);
            const real *ap = a + (p1 * n + p2) * n;
            const real *bq = b + (q1 * n + q2) * n;
            for (int p3 = 0; p3 < n; ++p3) acc += ap[p3] * bq[wrap(l3 - p3, n)];
          }
        }
        y[(l1 * n + l2) * n + l3] = acc;
      }
}

static real knorm(int n, int c1, int c2, int c3) {
  real a = cen(c1, n), b = cen(c2, n), c = cen(c3, n);
  return sqrt(a * a + b * b + c * c);
}

int SUFFIX(lbo_direct_linearized)(int n, double L, int J, const double *gj, const double *wj,
                          const double *Bj, double rho, const double *u, double theta,
                          int cutoff, double eps, const double *f, double *out) {
  const int n3 = n * n * n;
  const real h = 2.0 * L / n;
  real *M = malloc(sizeof(real) * n3), *Mg = malloc(sizeof(real) * n3);
  real *Mh = malloc(sizeof(real) * n3), *r = malloc(sizeof(real) * n3);
  real *mult = malloc(sizeof(real) * n3), *phit = malloc(sizeof(real) * n3);
  real *uj = malloc(sizeof(real) * n3), *psi = malloc(sizeof(real) * n3);
  real *tmp = malloc(sizeof(real) * n3), *Lp = calloc(n3, sizeof(real));
  real *Om = malloc(sizeof(real) * n3), *c1v = malloc(sizeof(real) * n3);
  real *c2v = malloc(sizeof(real) * n3);
  if (!M || !Mg || !Mh || !r || !mult || !phit || !uj || !psi || !tmp || !Lp || !Om || !c1v || !c2v)
    return 1;
  real *fr = malloc(sizeof(real) * n3);
  if (!fr) return 1;
  for (int i = 0; i < n3; ++i) fr[i] = f[i];
  /* the cut-off decision in double, exactly as the reading states it */
  const double hd = 2.0 * L / n;
  const double thresh = log(1.0 / eps) - 1.5 * log(2.0 * M_PI * theta);
  const real th = theta;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        int i = (a * n + b) * n + c;
        double w1 = cen(a, n) * hd, w2 = cen(b, n) * hd, w3 = cen(c, n) * hd;
        double d2d = (w1 - u[0]) * (w1 - u[0]) + (w2 - u[1]) * (w2 - u[1]) + (w3 - u[2]) * (w3 - u[2]);
        real v1 = cen(a, n) * h, v2 = cen(b, n) * h, v3 = cen(c, n) * h;
        real d2 = (v1 - u[0]) * (v1 - u[0]) + (v2 - u[1]) * (v2 - u[1]) + (v3 - u[2]) * (v3 - u[2]);
        real z2 = v1 * v1 + v2 * v2 + v3 * v3;
        M[i] = rho * pow(2 * PI_R * th, (real)-1.5) * exp(-d2 / (2 * th));
        Mg[i] = rho * pow(PI_R * th, (real)-1.5) * exp(-z2 / th);
        Mh[i] = rho * pow(PI_R * th, (real)-1.5) * exp(-d2 / th);
        r[i] = (cutoff && d2d / (2.0 * theta) > thresh) ? 0 : fr[i] / M[i];
      }
  for (int j = 0; j < J; ++j) {
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c)
          mult[(a * n + b) * n + c] = sincd(PI_R * gj[j] * knorm(n, a, b, c) / (2.0 * L));
    idft_even(n, mult, phit);
    for (int i = 0; i < n3; ++i) uj[i] = Mg[i] * phit[i];
    cyc_conv(n, uj, r, psi);
    for (int i = 0; i < n3; ++i) psi[i] *= Mh[i];
    cyc_conv(n, phit, psi, tmp);
    const real cj = 4.0 * PI_R * PI_R * wj[j] * Bj[j];
    for (int i = 0; i < n3; ++i) Lp[i] += cj * tmp[i];
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        real kn = knorm(n, a, b, c), acc = 0.0;
        for (int j = 0; j < J; ++j) acc += wj[j] * Bj[j] * sincd(PI_R * gj[j] * kn / L);
        mult[(a * n + b) * n + c] = 16.0 * PI_R * PI_R * acc;
      }
  idft_even(n, mult, Om);
  cyc_conv(n, Om, fr, c1v);
  cyc_conv(n, Om, M, c2v);
  for (int i = 0; i < n3; ++i) out[i] = (double)(Lp[i] - (M[i] * c1v[i] + fr[i] * c2v[i]));
  free(M); free(Mg); free(Mh); free(r); free(mult); free(phit); free(uj); free(psi);
  free(tmp); free(Lp); free(Om); free(c1v); free(c2v); free(fr);
  return 0;
}

/* Direct DFT, F[k] = sum_l x[l] exp(-2 pi i k.l / n) (sign s = -1) or the
 * inverse with 1/n^3 (s = +1).  Real/imag parts separate. */
static void dft_direct(int n, const real *xr, const real *xi, real *Fr, real *Fi, int s) {
  const int n3 = n * n * n;
  real *ct = malloc(sizeof(real) * n), *st = malloc(sizeof(real) * n);
  for (int t = 0; t < n; ++t) { ct[t] = cos(2.0 * PI_R * t / n); st[t] = sin(2.0 * PI_R * t / n); }
  for (int k1 = 0; k1 < n; ++k1)
    for (int k2 = 0; k2 < n; ++k2)
      for (int k3 = 0; k3 < n; ++k3) {
        real ar = 0.0, ai = 0.0;
        for (int l1 = 0; l1 < n; ++l1)
          for (int l2 = 0; l2 < n; ++l2)
            for (int l3 = 0; l3 < n; ++l3) {
              int t = (k1 * l1 + k2 * l2 + k3 * l3) % n;
              int idx = (l1 * n + l2) * n + l3;
              real c = ct[t], sn = s * st[t];
              real re = xr[idx], im = xi ? xi[idx] : 0.0;
              ar += re * c - im * sn;
              ai += re * sn + im * c;
            }
        int o = (k1 * n + k2) * n + k3;
        Fr[o] = s > 0 ? ar / n3 : ar;
        Fi[o] = s > 0 ? ai / n3 : ai;
      }
  free(ct); free(st);
}

/* per-dimension factor of the Nyquist-averaged multiplier exp(i alpha_d k) */
static void mfac(int n, real alpha, int c, real *re, real *im) {
  int k = cen(c, n);
  if (k == -(n / 2)) { *re = cos(alpha * (n / 2)); *im = 0.0; return; }
  *re = cos(alpha * k); *im = sin(alpha * k);
}

int SUFFIX(lbo_direct_quadratic)(int n, double L, int J, const double *gj, const double *wj,
                         const double *Bj, int M, const double *sig, const double *wm,
                         const double *f, const double *g, double *out) {
  const int n3 = n * n * n;
  real *Fr = malloc(sizeof(real) * n3), *Fi = malloc(sizeof(real) * n3);
  real *Gr = malloc(sizeof(real) * n3), *Gi = malloc(sizeof(real) * n3);
  real *Cr = malloc(sizeof(real) * n3), *Ci = malloc(sizeof(real) * n3); /* E(k) */
  real *Qr = calloc(n3, sizeof(real)), *Qi = calloc(n3, sizeof(real));
  real *qr = malloc(sizeof(real) * n3), *qi = malloc(sizeof(real) * n3);
  real *mult = malloc(sizeof(real) * n3), *Om = malloc(sizeof(real) * n3);
  real *t1 = malloc(sizeof(real) * n3), *t2 = malloc(sizeof(real) * n3);
  real *fr = malloc(sizeof(real) * n3), *gr = malloc(sizeof(real) * n3);
  if (!Fr || !Fi || !Gr || !Gi || !Cr || !Ci || !Qr || !Qi || !qr || !qi || !mult || !Om || !t1 || !t2 || !fr || !gr)
    return 1;
  const int bil = g != NULL;
  for (int i = 0; i < n3; ++i) {
    fr[i] = f[i];
    gr[i] = bil ? g[i] : 0;
  }
  dft_direct(n, fr, NULL, Fr, Fi, -1);
  if (bil) dft_direct(n, gr, NULL, Gr, Gi, -1);
  for (int j = 0; j < J; ++j)
    for (int m = 0; m < M; ++m) {
      real al[3];
      for (int d = 0; d < 3; ++d) al[d] = PI_R * gj[j] * sig[3 * m + d] / (2.0 * L);
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
          for (int c = 0; c < n; ++c) {
            real r1, i1, r2, i2, r3, i3;
            mfac(n, al[0], a, &r1, &i1); mfac(n, al[1], b, &r2, &i2); mfac(n, al[2], c, &r3, &i3);
            real pr = r1 * r2 - i1 * i2, pi = r1 * i2 + i1 * r2;
            int o = (a * n + b) * n + c;
            Cr[o] = pr * r3 - pi * i3;
            Ci[o] = pr * i3 + pi * r3;
          }
      const real wjm = wj[j] * wm[m] * Bj[j];
      for (int k1 = 0; k1 < n; ++k1)
        for (int k2 = 0; k2 < n; ++k2)
          for (int k3 = 0; k3 < n; ++k3) {
            real ir = 0.0, ii = 0.0;
            for (int l1 = 0; l1 < n; ++l1)
              for (int l2 = 0; l2 < n; ++l2)
                for (int l3 = 0; l3 < n; ++l3) {
                  int l = (l1 * n + l2) * n + l3;
                  int q = (wrap(k1 - l1, n) * n + wrap(k2 - l2, n)) * n + wrap(k3 - l3, n);
                  /* cos(a.(k-l)) cos(a.l) + sin(a.(k-l)) sin(a.l) */
                  real w = Cr[q] * Cr[l] + Ci[q] * Ci[l];
                  real xr, xi;
                  if (bil) {
                    xr = Fr[q] * Gr[l] - Fi[q] * Gi[l] + Gr[q] * Fr[l] - Gi[q] * Fi[l];
                    xi = Fr[q] * Gi[l] + Fi[q] * Gr[l] + Gr[q] * Fi[l] + Gi[q] * Fr[l];
                  } else {
                    xr = Fr[q] * Fr[l] - Fi[q] * Fi[l];
                    xi = Fr[q] * Fi[l] + Fi[q] * Fr[l];
                  }
                  ir += w * xr;
                  ii += w * xi;
                }
            int o = (k1 * n + k2) * n + k3;
            real s = sincd(PI_R * gj[j] * knorm(n, k1, k2, k3) / (2.0 * L));
            Qr[o] += wjm * s * ir / n3;
            Qi[o] += wjm * s * ii / n3;
          }
    }
  dft_direct(n, Qr, Qi, qr, qi, +1);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        real kn = knorm(n, a, b, c), acc = 0.0;
        for (int j = 0; j < J; ++j) acc += wj[j] * Bj[j] * sincd(PI_R * gj[j] * kn / L);
        mult[(a * n + b) * n + c] = 16.0 * PI_R * PI_R * acc;
      }
  idft_even(n, mult, Om);
  if (bil) {
    cyc_conv(n, Om, gr, t1);
    cyc_conv(n, Om, fr, t2);
    for (int i = 0; i < n3; ++i) out[i] = (double)(16 * PI_R * PI_R * qr[i] - (fr[i] * t1[i] + gr[i] * t2[i]));
  } else {
    cyc_conv(n, Om, fr, t1);
    for (int i = 0; i < n3; ++i) out[i] = (double)(16 * PI_R * PI_R * qr[i] - fr[i] * t1[i]);
  }
  free(Fr); free(Fi); free(Gr); free(Gi); free(Cr); free(Ci); free(Qr); free(Qi);
  free(qr); free(qi); free(mult); free(Om); free(t1); free(t2); free(fr); free(gr);
  return 0;
}
