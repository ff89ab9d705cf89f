// C entry points around the block-FGMRES host algebra (paper_2203_11025_gb300/csrc/block_ls.h)
// for the CPU tests: complex arrays are interleaved (re, im) doubles.
#include <complex>
#include <vector>

#include "block_ls.h"

using helm::cd;

static std::vector<cd> load(const double* a, size_t n) {
  std::vector<cd> v(n);
  for (size_t i = 0; i < n; ++i) v[i] = cd(a[2 * i], a[2 * i + 1]);
  return v;
}
static void store(const std::vector<cd>& v, double* a) {
  for (size_t i = 0; i < v.size(); ++i) { a[2 * i] = v[i].real(); a[2 * i + 1] = v[i].imag(); }
}

extern "C" {

// G (p x p, row-major) -> R, Rinv (p x p, row-major)
void chol_upper_c(const double* G, int p, double* R, double* Rinv) {
  std::vector<cd> r, ri;
  helm::chol_upper(load(G, (size_t)p * p), p, r, ri);
  store(r, R);
  store(ri, Rinv);
}

// S (p x p), Hbar ((m+1)p x mp, row-major); est (m x p): residual estimates after each block
// step; Y (mp x p, row-major): the least-squares solution after m steps
void block_ls_run(int p, int m, const double* S, const double* Hbar, double* est, double* Y) {
  helm::BlockLS ls;
  ls.reset(p, m, load(S, (size_t)p * p));
  const std::vector<cd> Hb = load(Hbar, (size_t)(m + 1) * p * m * p);
  for (int j = 0; j < m; ++j) {
    std::vector<cd> hb((size_t)(j + 2) * p * p);
    for (int r = 0; r < (j + 2) * p; ++r)
      for (int k = 0; k < p; ++k) hb[(size_t)r * p + k] = Hb[(size_t)r * m * p + j * p + k];
    const std::vector<double> e = ls.add(j, hb);
    for (int k = 0; k < p; ++k) est[j * p + k] = e[k];
  }
  store(ls.solve(m), Y);
}

}  // extern "C"
