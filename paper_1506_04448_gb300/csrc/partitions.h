// Compile-time term table of the order-p sketched contractions (orderp.cu): plain constexpr
// C++17, no CUDA, so that host code (and a host-compiled test) can evaluate it too.
//
// For the partitions lambda of P (z_lambda = prod_k k^{m_k} m_k!, m_k the multiplicity of part k):
//   target 0: a term 1/z_lambda of Y over all of lambda's parts, for every lambda other than (P);
//   target k in 1..P-1: a term m_k(lambda)/z_lambda of F R_k over lambda's other parts, for every
//   lambda containing the part k.
#pragma once

namespace tsk {

constexpr int kMaxOrder = 6;
constexpr int kMaxTerms = 48;

// The table for order P (the kernel unrolls it, so every product is a chain of complex
// multiplications on fixed registers).  Partitions of P are enumerated in reverse lexicographic
// order by the classic successor rule: strip trailing ones, decrement the last part above one,
// refill with copies of it and the remainder.
template <int P>
struct CTerms {
  float coef[kMaxTerms];
  int target[kMaxTerms];
  int nparts[kMaxTerms];
  int parts[kMaxTerms][kMaxOrder];
  int count;
};

template <int P>
constexpr CTerms<P> compile_terms() {
  CTerms<P> out{};
  out.count = 0;
  int a[kMaxOrder + 1] = {};
  int len = 1;
  a[0] = P;
  while (true) {
    // z_lambda = prod_k k^{m_k} m_k! for the partition a[0..len)
    int mult[kMaxOrder + 1] = {};
    for (int j = 0; j < len; ++j) ++mult[a[j]];
    long long z = 1;
    for (int k = 1; k <= P; ++k)
      for (int j = 1; j <= mult[k]; ++j) z *= (long long)k * j;
    if (!(len == 1 && a[0] == P)) {
      out.coef[out.count] = 1.0f / (float)z;
      out.target[out.count] = 0;
      out.nparts[out.count] = len;
      for (int j = 0; j < len; ++j) out.parts[out.count][j] = a[j];
      ++out.count;
    }
    for (int k = 1; k < P; ++k) {
      if (mult[k] == 0) continue;
      out.coef[out.count] = (float)mult[k] / (float)z;
      out.target[out.count] = k;
      int c = 0;
      bool dropped = false;
      for (int j = 0; j < len; ++j) {
        if (!dropped && a[j] == k) {
          dropped = true;
          continue;
        }
        out.parts[out.count][c++] = a[j];
      }
      out.nparts[out.count] = c;
      ++out.count;
    }
    int rem = 0;
    while (len > 0 && a[len - 1] == 1) {
      ++rem;
      --len;
    }
    if (len == 0) break;
    a[len - 1] -= 1;
    ++rem;
    const int x = a[len - 1];
    while (rem > x) {
      a[len++] = x;
      rem -= x;
    }
    a[len++] = rem;
  }
  return out;
}

template <int P>
struct TermTable {
  static constexpr CTerms<P> value = compile_terms<P>();
};

}  // namespace tsk
