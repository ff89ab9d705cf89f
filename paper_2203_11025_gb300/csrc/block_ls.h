// Host dense algebra of block flexible GMRES (the CPU solver of Sec. 4): the Cholesky QR
// factor of a block's Gram matrix with dependent columns, and the block least-squares
// problem min ||E_1 S - Hbar Y|| reduced by Householder reflections one block column at a
// time.  Plain C++ (FP64 complex): the solver includes it, and the CPU tests compile it
// alone.
#pragma once
#include <cmath>
#include <complex>
#include <vector>

namespace helm {

typedef std::complex<double> cd;

// G = R^H R for the Hermitian p x p Gram matrix G (row-major); R upper triangular.  A
// pivot below 1e-12 of its column's squared norm marks a column that depends on the
// previous ones: its row of R is zero, and column k of Rinv (the inverse of R on the
// independent columns) is zero, so W Rinv has a zero column there and W = (W Rinv) R.
inline void chol_upper(const std::vector<cd>& G, int p, std::vector<cd>& R, std::vector<cd>& Rinv) {
  R.assign((size_t)p * p, cd(0));
  Rinv.assign((size_t)p * p, cd(0));
  std::vector<char> dep(p, 0);
  for (int j = 0; j < p; ++j) {
    double d = G[(size_t)j * p + j].real();
    for (int i = 0; i < j; ++i) d -= std::norm(R[(size_t)i * p + j]);
    if (!(d > 1e-12 * G[(size_t)j * p + j].real())) { dep[j] = 1; continue; }
    const double rjj = std::sqrt(d);
    R[(size_t)j * p + j] = rjj;
    for (int k = j + 1; k < p; ++k) {
      cd t = G[(size_t)j * p + k];
      for (int i = 0; i < j; ++i) t -= std::conj(R[(size_t)i * p + j]) * R[(size_t)i * p + k];
      R[(size_t)j * p + k] = t / rjj;
    }
  }
  for (int k = 0; k < p; ++k) {
    if (dep[k]) continue;
    for (int i = k; i >= 0; --i) {
      if (dep[i]) continue;
      cd t = i == k ? cd(1) : cd(0);
      for (int l = i + 1; l <= k; ++l) t -= R[(size_t)i * p + l] * Rinv[(size_t)l * p + k];
      Rinv[(size_t)i * p + k] = t / R[(size_t)i * p + i];
    }
  }
}

// Least squares of block FGMRES: Hbar ((m+1)p x mp, block upper Hessenberg with upper
// triangular subdiagonal blocks) reduced to upper triangular form by one Householder
// reflection per column (column c touches rows c .. c + p), applied to g = Q^H E_1 S too.
struct BlockLS {
  int p = 0, m = 0, rows = 0;
  std::vector<cd> H;      // column-major, rows x (m p)
  std::vector<cd> g;      // column-major, rows x p
  std::vector<cd> refl;   // reflector of column c: p + 1 entries
  void reset(int p_, int m_, const std::vector<cd>& S) {
    p = p_; m = m_; rows = (m + 1) * p;
    H.assign((size_t)rows * m * p, cd(0));
    g.assign((size_t)rows * p, cd(0));
    refl.assign((size_t)m * p * (p + 1), cd(0));
    for (int i = 0; i < p; ++i)
      for (int k = 0; k < p; ++k) g[(size_t)k * rows + i] = S[(size_t)i * p + k];
  }
  cd& h(int r, int c) { return H[(size_t)c * rows + r]; }
  // col <- (I - 2 v v^H) col on rows c .. c + p (reflector of column c)
  void apply(int c, cd* col) {
    const cd* v = &refl[(size_t)c * (p + 1)];
    cd t = 0;
    for (int i = 0; i <= p; ++i) t += std::conj(v[i]) * col[c + i];
    for (int i = 0; i <= p; ++i) col[c + i] -= 2.0 * v[i] * t;
  }
  // Block column j (rows 0 .. (j+2)p - 1 of Hbar, row-major hb[(j+2)p][p]); returns the
  // least-squares residual norm of each right-hand side after j + 1 block steps.
  std::vector<double> add(int j, const std::vector<cd>& hb) {
    const int c0 = j * p;
    for (int k = 0; k < p; ++k)
      for (int r = 0; r < (j + 2) * p; ++r) h(r, c0 + k) = hb[(size_t)r * p + k];
    for (int c = 0; c < c0; ++c)
      for (int k = 0; k < p; ++k) apply(c, &H[(size_t)(c0 + k) * rows]);
    for (int t = 0; t < p; ++t) {
      const int c = c0 + t;
      cd* x = &H[(size_t)c * rows];
      double sig = 0;
      for (int i = 0; i <= p; ++i) sig += std::norm(x[c + i]);
      sig = std::sqrt(sig);
      cd* v = &refl[(size_t)c * (p + 1)];
      if (sig == 0.0) {
        for (int i = 0; i <= p; ++i) v[i] = 0;
        continue;
      }
      const cd ph = std::abs(x[c]) > 0 ? x[c] / std::abs(x[c]) : cd(1);
      const cd alpha = -ph * sig;
      for (int i = 0; i <= p; ++i) v[i] = x[c + i];
      v[0] -= alpha;
      double vn = 0;
      for (int i = 0; i <= p; ++i) vn += std::norm(v[i]);
      vn = std::sqrt(vn);
      for (int i = 0; i <= p; ++i) v[i] /= vn;
      for (int k = t; k < p; ++k) apply(c, &H[(size_t)(c0 + k) * rows]);
      for (int k = 0; k < p; ++k) apply(c, &g[(size_t)k * rows]);
    }
    std::vector<double> est(p);
    for (int k = 0; k < p; ++k) {
      double e = 0;
      for (int r = (j + 1) * p; r < (j + 2) * p; ++r) e += std::norm(g[(size_t)k * rows + r]);
      est[k] = std::sqrt(e);
    }
    return est;
  }
  // Y = R^-1 g over the first n = (j+1) p rows (row-major n x p); zero where R is singular.
  std::vector<cd> solve(int nblk) {
    const int n = nblk * p;
    std::vector<cd> Y((size_t)n * p, cd(0));
    for (int k = 0; k < p; ++k)
      for (int i = n - 1; i >= 0; --i) {
        cd t = g[(size_t)k * rows + i];
        for (int l = i + 1; l < n; ++l) t -= h(i, l) * Y[(size_t)l * p + k];
        const cd d = h(i, i);
        Y[(size_t)i * p + k] = std::abs(d) > 1e-300 ? t / d : cd(0);
      }
    return Y;
  }
};

}  // namespace helm
