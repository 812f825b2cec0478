// Host 1D tables: Gauss-Legendre rule, GLL nodes, Lagrange basis, and the
// even-odd split of N^1D, (N^1D)^T, D~^1D, (D~^1D)^T (Sec. 3.2; Sec. 5.4).
// Nodes come from Newton's method on Legendre polynomials (three-term
// recurrence), written here independently of any other component.
#include <cmath>
#include <cstring>

#include "fe_ks_internal.h"

namespace feks {

// P_n(x) and P_n'(x) by the Bonnet recurrence.
static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  if (std::fabs(std::fabs(x) - 1.0) < 1e-300) {
    *dP = (x > 0 ? 1.0 : ((n - 1) % 2 ? -1.0 : 1.0)) * n * (n + 1) / 2.0;
  } else {
    *dP = n * (p0 - x * p1) / (1.0 - x * x);
  }
}

void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, z, &P, &dP);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(n, z, &P, &dP);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

void gauss_lobatto(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  const int p = n - 1;
  x[0] = -1.0;
  x[n - 1] = 1.0;
  for (int i = 1; i < n - 1; ++i) {
    double z = -std::cos(pi * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, z, &P, &dP);
      // Legendre's equation gives P'' = (2 z P' - p(p+1) P) / (1 - z^2)
      double d2 = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
      double dz = dP / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre(p, x[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

// Lagrange basis on `nodes`: val[i] = L_i(x), der[i] = L_i'(x) (product rule).
void lagrange_eval(int n, const double* nodes, double x, double* val, double* der) {
  for (int i = 0; i < n; ++i) {
    double v = 1.0, d = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double f = 1.0 / (nodes[i] - nodes[j]);
      d = d * (x - nodes[j]) * f + v * f;
      v *= (x - nodes[j]) * f;
    }
    val[i] = v;
    der[i] = d;
  }
}

template <typename T>
static void split(const double* M, int NO, int NI, EOMat<T>* out) {
  *out = EOMat<T>{};
  const int HO = NO / 2, HI = NI / 2;
  for (int o = 0; o < HO; ++o) {
    for (int i = 0; i < HI; ++i) {
      out->E[o][i] = (T)(0.5 * (M[o * NI + i] + M[o * NI + NI - 1 - i]));
      out->O[o][i] = (T)(0.5 * (M[o * NI + i] - M[o * NI + NI - 1 - i]));
    }
    if (NI % 2) out->E[o][HI] = (T)M[o * NI + HI];
  }
  if (NO % 2)
    for (int i = 0; i <= HI && i < NI; ++i) out->MID[i] = (T)M[HO * NI + i];
}

template <typename T>
void build_eo_tables(int p, int nq, EOTables<T>* out) {
  const int np = p + 1;
  double xg[kMaxN], wg[kMaxN], xq[kMaxN], wq[kMaxN];
  gauss_lobatto(np, xg, wg);
  gauss_legendre(nq, xq, wq);
  double N[kMaxN * kMaxN], Nt[kMaxN * kMaxN], D[kMaxN * kMaxN], Dt[kMaxN * kMaxN];
  double val[kMaxN], der[kMaxN];
  for (int q = 0; q < nq; ++q) {
    lagrange_eval(np, xg, xq[q], val, der);
    for (int i = 0; i < np; ++i) {
      N[q * np + i] = val[i];
      Nt[i * nq + q] = val[i];
    }
    lagrange_eval(nq, xq, xq[q], val, der);
    for (int r = 0; r < nq; ++r) {
      D[q * nq + r] = der[r];
      Dt[r * nq + q] = der[r];
    }
  }
  split<T>(N, nq, np, &out->N);
  split<T>(Nt, np, nq, &out->Nt);
  split<T>(D, nq, nq, &out->D);
  split<T>(Dt, nq, nq, &out->Dt);
}

template <>
void build_eo_tables<ff2>(int p, int nq, EOTables<ff2>* out) {
  EOTables<double> d;
  build_eo_tables<double>(p, nq, &d);
  const double* src = reinterpret_cast<const double*>(&d);
  ff2* dst = reinterpret_cast<ff2*>(out);
  static_assert(sizeof(EOTables<double>) == sizeof(EOTables<ff2>), "table layouts differ");
  for (size_t i = 0; i < sizeof(EOTables<double>) / sizeof(double); ++i) dst[i] = ff_from_double_host(src[i]);
}

// Round to the nearest BF16 (ties to even) through the nearest float.
uint16_t bf16_bits(double x) {
  const float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Nearest FP16 (ties to even) of a value inside the FP16 range, through the
// nearest float; subnormal results are rounded at their fixed quantum 2^-24.
uint16_t f16_bits(double x) {
  const float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t sign = (u >> 16) & 0x8000u;
  const int e = (int)((u >> 23) & 0xFFu) - 127;
  uint32_t mant = u & 0x7FFFFFu;
  if (e > 15) return (uint16_t)(sign | 0x7C00u);                 // beyond the range: infinity
  if (e < -25 || (u & 0x7FFFFFFFu) == 0) return (uint16_t)sign;  // below half the smallest subnormal
  if (e < -14) {                                                  // subnormal: quantum 2^-24
    mant |= 0x800000u;
    const int sh = -e - 1;   // value = mant 2^(e - 23) = (mant >> sh) quanta of 2^-24
    const uint32_t q = mant >> (sh);
    const uint32_t rem = mant & ((1u << sh) - 1u), half = 1u << (sh - 1);
    const uint32_t r = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
    return (uint16_t)(sign | r);
  }
  uint32_t h = ((uint32_t)(e + 15) << 10) | (mant >> 13);
  const uint32_t rem = mant & 0x1FFFu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;   // carries into the exponent correctly
  return (uint16_t)(sign | h);
}

// Remainder of the BF16 split: the nearest BF16 of x - (nearest BF16 of x), as
// its bit pattern (hi + lo then carries about 16 significant bits of x).
uint16_t bf16_lo_bits(double x) {
  const uint32_t h = (uint32_t)bf16_bits(x) << 16;
  float hv;
  std::memcpy(&hv, &h, 4);
  return bf16_bits(x - (double)hv);
}

void build_tc_frags(int p, uint32_t* out, int kind) {
  const int n = p + 1;
  double xg[kMaxN], wg[kMaxN], xq[kMaxN], wq[kMaxN], val[kMaxN], der[kMaxN];
  gauss_lobatto(n, xg, wg);
  gauss_legendre(n, xq, wq);
  double Nm[kMaxN][kMaxN], Dm[kMaxN][kMaxN];   // [q][i]
  for (int q = 0; q < n; ++q) {
    lagrange_eval(n, xg, xq[q], val, der);
    for (int i = 0; i < n; ++i) {
      Nm[q][i] = val[i];
      Dm[q][i] = der[i];
    }
  }
  // B[k][col] of each op (K x N operand of D = A B; zero outside n x n)
  auto B = [&](int op, int k, int col) -> double {
    if (k >= n || col >= n) return 0.0;
    switch (op) {
      case 0: return Nm[col][k];   // forward: k = node, col = Gauss point
      case 1: return Dm[col][k];
      case 2: return Nm[k][col];   // transposed: k = Gauss point, col = node
      default: return Dm[k][col];
    }
  };
  for (int op = 0; op < 4; ++op)
    for (int tile = 0; tile < 2; ++tile)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane / 4, t = lane % 4, col = 8 * tile + g;
        for (int r = 0; r < 2; ++r) {
          const int k = 2 * t + 8 * r;
          auto h = [&](double x) -> uint32_t {
            return kind == 1 ? f16_bits(x) : kind == 2 ? bf16_lo_bits(x) : bf16_bits(x);
          };
          out[((op * 2 + tile) * 32 + lane) * 2 + r] = h(B(op, k, col)) | (h(B(op, k + 1, col)) << 16);
        }
      }
}

template void build_eo_tables<double>(int, int, EOTables<double>*);
template void build_eo_tables<float>(int, int, EOTables<float>*);

}  // namespace feks
