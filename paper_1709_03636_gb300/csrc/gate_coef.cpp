// Leaf tensors (the gate, state, observable and channel tensors of Section 2)
// as per-element coefficients.  Every element of every leaf kind is
//   A cos(t/2) + B sin(t/2) + C,   t = constant + coeff * params[slot],
// with complex A, B, C fixed by the kind (and conjugated on the bra side), so
// its derivative with respect to params[slot] is
//   coeff (B/2) cos(t/2) - coeff (A/2) sin(t/2).
// The warp executor builds its gate table from these records: one sine and
// cosine per gate, then one complex multiply-add per element, the same code
// for every kind.  Element index bit k is the leaf's label k (as in the
// executors' closed forms).
#include <cmath>
#include <complex>
#include <cstring>

#include "qtc_internal.h"

namespace qtc {

using cd = std::complex<double>;

void gate_coefficients(const GateSpec& s, cd* A, cd* B, cd* C) {
  const int n = 1 << leaf_rank_of(s.kind);
  for (int i = 0; i < n; ++i) A[i] = B[i] = C[i] = 0.0;
  const double r = 0.70710678118654752440;
  const cd I(0.0, 1.0);
  switch (s.kind) {
    case LK_ZERO: case LK_PROJ0: C[0] = 1.0; break;
    case LK_PROJ1: C[1] = 1.0; break;
    case LK_PLUS: C[0] = r; C[1] = r; break;
    case LK_ZDIAG: C[0] = 1.0; C[1] = -1.0; break;
    case LK_H:
      for (int i = 0; i < 4; ++i) C[i] = (i == 3) ? -r : r;
      break;
    case LK_X: case LK_OBS_X: C[1] = 1.0; C[2] = 1.0; break;
    case LK_Y: case LK_OBS_Y: C[2] = -I; C[1] = I; break;   // [out][in]: [0][1] = -i
    case LK_Z: case LK_OBS_Z: C[0] = 1.0; C[3] = -1.0; break;
    case LK_RX:  // cos(t/2) I - i sin(t/2) X
      A[0] = A[3] = 1.0;
      B[1] = B[2] = -I;
      break;
    case LK_RZ: case LK_RZDIAG: {  // diag(exp(-i t/2), exp(+i t/2))
      const int i1 = s.kind == LK_RZ ? 3 : 1;
      A[0] = 1.0;
      B[0] = -I;
      A[i1] = 1.0;
      B[i1] = I;
      break;
    }
    case LK_ZZDIAG: case LK_ZZ:  // exp(-i z_a z_b t/2)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const double zz = (a == b) ? 1.0 : -1.0;
          const int idx = s.kind == LK_ZZDIAG ? (a | b << 1) : (a | b << 1 | a << 2 | b << 3);
          A[idx] = 1.0;
          B[idx] = -I * zz;
        }
      break;
    case LK_CNOT:
      for (int c = 0; c < 2; ++c)
        for (int t = 0; t < 2; ++t) C[c | (t ^ c) << 1 | c << 2 | t << 3] = 1.0;
      break;
    case LK_OBS_I: C[0] = 1.0; C[3] = 1.0; break;
    case LK_ONES: C[0] = 1.0; C[1] = 1.0; break;
    case LK_OBS_P0: C[0] = 1.0; break;
    case LK_OBS_P1: C[3] = 1.0; break;
    case LK_CNOTX:  // [t_out, c, t_in]: 1 where t_out = t_in xor c
      for (int i = 0; i < 8; ++i) C[i] = ((i & 1) == (((i >> 1) ^ (i >> 2)) & 1)) ? 1.0 : 0.0;
      break;
    case LK_DEPOL: case LK_DEPHASE: case LK_AMPDAMP: {
      // sum_k K[ko][ki] conj(K[bo][bi]) at ko | bo<<1 | ki<<2 | bi<<3 (strength
      // = constant): depolarizing (1-s) I(x)I + s/3 (XX* + YY* + ZZ*), dephasing
      // (1-s) I(x)I + s ZZ*, amplitude damping K0 K0* + K1 K1*
      const double st = s.constant;
      for (int i = 0; i < 16; ++i) {
        const int ko = i & 1, bo = (i >> 1) & 1, ki = (i >> 2) & 1, bi = (i >> 3) & 1;
        const bool keep = ko == ki && bo == bi;
        const double zz = (ko ^ bo) ? -1.0 : 1.0;
        double v = 0.0;
        if (s.kind == LK_DEPOL) {
          if (keep) v = (1.0 - st) + st / 3.0 * zz;
          else if (ko != ki && bo != bi && ko == bo) v = 2.0 * st / 3.0;
        } else if (s.kind == LK_DEPHASE) {
          if (keep) v = (1.0 - st) + st * zz;
        } else {
          if (keep) v = (ko ? std::sqrt(1.0 - st) : 1.0) * (bo ? std::sqrt(1.0 - st) : 1.0);
          else if (ko == 0 && bo == 0 && ki == 1 && bi == 1) v = st;
        }
        C[i] = v;
      }
      break;
    }
    default:
      break;
  }
  if (s.conj)
    for (int i = 0; i < n; ++i) {
      A[i] = std::conj(A[i]);
      B[i] = std::conj(B[i]);
      C[i] = std::conj(C[i]);
    }
}

namespace {

template <typename Rec, typename R>
void put(std::vector<uint8_t>& out, uint32_t j, uint32_t gate, cd a, cd b, cd c) {
  Rec rec{};
  const R v[6] = {(R)a.real(), (R)a.imag(), (R)b.real(), (R)b.imag(), (R)c.real(), (R)c.imag()};
  std::memcpy(rec.a, v, sizeof v);
  rec.gate = gate;
  std::memcpy(out.data() + (size_t)j * sizeof(Rec), &rec, sizeof rec);
}

}  // namespace

std::vector<uint8_t> coefficient_table(const std::vector<GateEntryDev>& gates,
                                       uint32_t table_elems, int dtype) {
  const bool wide = dtype == QTC_C128;
  const size_t rec = wide ? sizeof(TabCoef64) : sizeof(TabCoef32);
  std::vector<uint8_t> out(rec * table_elems, 0);  // padding elements: zero
  cd A[16], B[16], C[16];
  for (size_t g = 0; g < gates.size(); ++g) {
    const GateSpec& s = gates[g].spec;
    gate_coefficients(s, A, B, C);
    const int n = 1 << leaf_rank_of(s.kind);
    for (int i = 0; i < n; ++i) {
      const uint32_t jv = gates[g].val_off + i;
      if (wide) put<TabCoef64, double>(out, jv, (uint32_t)g, A[i], B[i], C[i]);
      else put<TabCoef32, float>(out, jv, (uint32_t)g, A[i], B[i], C[i]);
      if (s.slot >= 0) {
        const uint32_t jd = gates[g].der_off + i;
        const cd da = 0.5 * s.coeff * B[i], db = -0.5 * s.coeff * A[i];
        if (wide) put<TabCoef64, double>(out, jd, (uint32_t)g, da, db, 0.0);
        else put<TabCoef32, float>(out, jd, (uint32_t)g, da, db, 0.0);
      }
    }
  }
  return out;
}

void leaf_values(const GateSpec& s, const double* params, double* val, double* der) {
  cd A[16], B[16], C[16];
  gate_coefficients(s, A, B, C);
  const double t = s.constant + (s.slot >= 0 ? s.coeff * params[s.slot] : 0.0);
  const double c = std::cos(0.5 * t), sn = std::sin(0.5 * t);
  const int n = 1 << leaf_rank_of(s.kind);
  for (int i = 0; i < n; ++i) {
    const cd v = A[i] * c + B[i] * sn + C[i];
    val[2 * i] = v.real();
    val[2 * i + 1] = v.imag();
    if (der) {
      const cd d = s.slot >= 0 ? s.coeff * (0.5 * B[i] * c - 0.5 * A[i] * sn) : cd(0.0);
      der[2 * i] = d.real();
      der[2 * i + 1] = d.imag();
    }
  }
}

}  // namespace qtc
