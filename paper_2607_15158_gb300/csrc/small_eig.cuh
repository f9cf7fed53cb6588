// Eigenvalues of a small dense complex matrix (m <= 32): Householder
// reduction to upper Hessenberg form, then the shifted QR algorithm with
// Wilkinson shifts, Givens bulge chasing and deflation of negligible
// subdiagonal entries (Golub & Van Loan, "Matrix Computations", 4th ed.,
// Alg. 7.4.2 and 7.5: the single-shift complex form). Written for one
// thread (the Rayleigh-Ritz matrices of the transfer-matrix spectrum are
// m x m with m ~ 8); usable on the host and the device.
#pragma once

#include <cmath>

namespace ctm {

struct zc {
  double re, im;
};
__host__ __device__ inline zc zmk(double r, double i) { return zc{r, i}; }
__host__ __device__ inline zc zadd(zc a, zc b) { return zc{a.re + b.re, a.im + b.im}; }
__host__ __device__ inline zc zsub(zc a, zc b) { return zc{a.re - b.re, a.im - b.im}; }
__host__ __device__ inline zc zmul(zc a, zc b) {
  return zc{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ inline zc zconj(zc a) { return zc{a.re, -a.im}; }
__host__ __device__ inline double zabs(zc a) { return hypot(a.re, a.im); }
__host__ __device__ inline zc zscale(zc a, double s) { return zc{a.re * s, a.im * s}; }
__host__ __device__ inline zc zdiv(zc a, zc b) {
  const double d = b.re * b.re + b.im * b.im;
  return zc{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// principal square root
__host__ __device__ inline zc zsqrt(zc a) {
  const double r = zabs(a);
  if (r == 0.0) return zc{0.0, 0.0};
  double x = sqrt(0.5 * (r + fabs(a.re)));
  double y = a.im / (2.0 * x);
  if (a.re < 0.0) {
    const double t = fabs(y);
    y = a.im >= 0.0 ? x : -x;
    x = t;
  }
  return zc{x, y};
}

// Eigenvalues of the m x m row-major matrix H (overwritten) into ev[m];
// returns the number of QR iterations, or -1 if some eigenvalue did not
// converge within 60 m iterations.
__host__ __device__ inline int small_eigvals(int m, zc* H, zc* ev) {
  // Householder reduction to upper Hessenberg form
  for (int k = 0; k + 2 < m; ++k) {
    double nx = 0.0;
    for (int i = k + 1; i < m; ++i) nx += H[i * m + k].re * H[i * m + k].re + H[i * m + k].im * H[i * m + k].im;
    nx = sqrt(nx);
    if (nx == 0.0) continue;
    const zc x0 = H[(k + 1) * m + k];
    const double a0 = zabs(x0);
    // v = x + phase(x0) |x| e_1, H <- (I - 2 v v^H / v^H v) H (I - ...)
    const zc ph = a0 > 0.0 ? zscale(x0, 1.0 / a0) : zc{1.0, 0.0};
    zc v[32];
    for (int i = k + 1; i < m; ++i) v[i] = H[i * m + k];
    v[k + 1] = zadd(v[k + 1], zscale(ph, nx));
    double vv = 0.0;
    for (int i = k + 1; i < m; ++i) vv += v[i].re * v[i].re + v[i].im * v[i].im;
    if (vv == 0.0) continue;
    for (int j = 0; j < m; ++j) {
      zc s = {0.0, 0.0};
      for (int i = k + 1; i < m; ++i) s = zadd(s, zmul(zconj(v[i]), H[i * m + j]));
      s = zscale(s, 2.0 / vv);
      for (int i = k + 1; i < m; ++i) H[i * m + j] = zsub(H[i * m + j], zmul(v[i], s));
    }
    for (int i = 0; i < m; ++i) {
      zc s = {0.0, 0.0};
      for (int j = k + 1; j < m; ++j) s = zadd(s, zmul(H[i * m + j], v[j]));
      s = zscale(s, 2.0 / vv);
      for (int j = k + 1; j < m; ++j) H[i * m + j] = zsub(H[i * m + j], zmul(s, zconj(v[j])));
    }
    for (int i = k + 2; i < m; ++i) H[i * m + k] = zc{0.0, 0.0};
  }
  // shifted QR iterations on the active window [lo, hi]
  const double eps = 2.220446049250313e-16;
  int hi = m - 1, iters = 0, since = 0;
  while (hi >= 0) {
    if (hi == 0) {
      ev[0] = H[0];
      break;
    }
    int l = hi;
    while (l > 0) {
      const double sc = zabs(H[l * m + l]) + zabs(H[(l - 1) * m + l - 1]);
      if (zabs(H[l * m + l - 1]) <= eps * (sc > 0.0 ? sc : 1.0)) break;
      --l;
    }
    if (l == hi) {
      ev[hi] = H[hi * m + hi];
      H[hi * m + hi - 1] = zc{0.0, 0.0};
      --hi;
      since = 0;
      continue;
    }
    if (iters > 60 * m) return -1;
    ++iters;
    ++since;
    // Wilkinson shift: eigenvalue of the trailing 2 x 2 closer to H[hi][hi]
    const zc a = H[(hi - 1) * m + hi - 1], b = H[(hi - 1) * m + hi], c = H[hi * m + hi - 1],
             d = H[hi * m + hi];
    const zc hd = zscale(zsub(a, d), 0.5);
    const zc disc = zsqrt(zadd(zmul(hd, hd), zmul(b, c)));
    const zc mid = zscale(zadd(a, d), 0.5);
    zc mu1 = zadd(mid, disc), mu2 = zsub(mid, disc);
    zc mu = zabs(zsub(mu1, d)) < zabs(zsub(mu2, d)) ? mu1 : mu2;
    if (since % 11 == 10) {
      // exceptional shift after a run without deflation
      mu = zadd(d, zscale(zc{zabs(c), 0.0}, 0.75));
    }
    // implicit single-shift step: Givens rotations chase the bulge
    zc x = zsub(H[l * m + l], mu), y = H[(l + 1) * m + l];
    for (int k = l; k < hi; ++k) {
      const double r = sqrt(x.re * x.re + x.im * x.im + y.re * y.re + y.im * y.im);
      if (r == 0.0) break;
      // G = [[cc, s], [-conj(s), cc]] with G [x; y] = [r; 0]
      const double ax = zabs(x);
      double cc;
      zc s;
      if (ax == 0.0) {
        cc = 0.0;
        s = zconj(zscale(y, 1.0 / zabs(y)));
      } else {
        cc = ax / r;
        const zc px = zscale(x, 1.0 / ax);
        s = zscale(zmul(px, zconj(y)), 1.0 / r);
      }
      const int j0 = k > l ? k - 1 : l;
      for (int j = j0; j <= hi; ++j) {
        const zc u = H[k * m + j], w = H[(k + 1) * m + j];
        H[k * m + j] = zadd(zscale(u, cc), zmul(s, w));
        H[(k + 1) * m + j] = zsub(zscale(w, cc), zmul(zconj(s), u));
      }
      const int i1 = k + 2 < hi ? k + 2 : hi;
      for (int i = l; i <= i1; ++i) {
        const zc u = H[i * m + k], w = H[i * m + k + 1];
        H[i * m + k] = zadd(zscale(u, cc), zmul(zconj(s), w));
        H[i * m + k + 1] = zsub(zscale(w, cc), zmul(s, u));
      }
      if (k + 1 < hi) {
        x = H[(k + 1) * m + k];
        y = H[(k + 2) * m + k];
      }
    }
  }
  return iters;
}

}  // namespace ctm
