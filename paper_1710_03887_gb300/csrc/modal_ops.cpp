// Operators of the paper's own discretisation (Appendix A): the weak form of
// Eq. 10 in the orthonormal basis of Eq. 11 (mass matrix J I), its volume
// integral by a Gauss rule of degree 2p and its surface integrals by one of
// degree 2p+1.
//
// The library keeps the state as nodal values of the same polynomial, so
// the scheme becomes fixed matrices on nodal values. With l_j the Lagrange
// basis of the nodes, M^-1 = V V^T the inverse reference mass matrix (V the
// orthonormal Vandermonde: the identity mass matrix of the modal form seen
// through the change of basis), D_a the nodal derivative matrices and the
// metric-folded fluxes G_a = sum_d (dr_a/dx_d) F_d at the volume points,
//   du_n/dt = sum_a sum_q Sv_a[n][q] G_a(x_q) - sum_f Fscale_f sum_q Sf_f[n][q] F*_q
//   Sv_a[n][q] = sum_j M^-1[n][j] (dl_j/dr_a)(x_q) w_q,  dl_j/dr_a (x_q) = sum_m l_m(x_q) D_a[m][j]
//   Sf_f[n][q] = sum_j M^-1[n][j] l_j(x_fq) wf_q
// and the traces at face points come from the face's nodal values,
// u(x_fq) = sum_m l_{Fmask[f][m]}(x_fq) u_{Fmask[f][m]} (the other Lagrange
// functions vanish on the face).
//
// Gauss rules: collapsed-coordinate products of n-point Gauss-Jacobi rules,
// n = floor(d/2) + 1 (exact to degree 2n - 1 >= d). Tetrahedron:
// r = (1+a)(1-b)(1-c)/4 - 1, s = (1+b)(1-c)/2 - 1, t = c with weights
// w_a w_b w_c / 8 (a: Legendre, b: Jacobi (1,0), c: Jacobi (2,0)); triangle
// (-1,-1), (1,-1), (-1,1): u = (1+a)(1-b)/2 - 1, v = b with w_a w_b / 2.
// Face f is the image of the triangle under its vertex triple with weights
// (-(u+v)/2, (1+u)/2, (1+v)/2). One point set per face: the element with
// the lower index uses its own rule (variant 0); its neighbour evaluates at
// the same physical points, the neighbour's rule seen through the
// orientation code o (variant 1 + o), so both integrate the same flux.
#include <algorithm>
#include <cmath>

#include "dg_host.hpp"

namespace dg {

namespace {

// Jacobi polynomial P_n^(alpha, 0)(x) (the standard normalisation, P_n(1) =
// binom(n + alpha, n)) and its derivative, by the three-term recurrence.
void jacobi_p(int n, double alpha, double x, double& P, double& dP) {
  auto eval = [](int m, double al, double be, double z) {
    if (m == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * ((al + be + 2.0) * z + (al - be));
    for (int k = 1; k < m; ++k) {
      const double s = 2.0 * k + al + be;
      const double a1 = 2.0 * (k + 1) * (k + al + be + 1) * s;
      const double a2 = (s + 1) * (al * al - be * be);
      const double a3 = s * (s + 1) * (s + 2);
      const double a4 = 2.0 * (k + al) * (k + be) * (s + 2);
      const double p2 = ((a2 + a3 * z) * p1 - a4 * p0) / a1;
      p0 = p1;
      p1 = p2;
    }
    return p1;
  };
  P = eval(n, alpha, 0.0, x);
  dP = n == 0 ? 0.0 : 0.5 * (n + alpha + 1.0) * eval(n - 1, alpha + 1.0, 1.0, x);
}

}  // namespace

void gauss_jacobi(int n, double alpha, double* x, double* w) {
  // Newton with deflation from the Chebyshev-Gauss points
  for (int k = 0; k < n; ++k) {
    double z = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * n));
    if (k > 0) z = 0.5 * (z + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double P, dP;
      jacobi_p(n, alpha, z, P, dP);
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += 1.0 / (z - x[j]);
      const double dz = P / (dP - s * P);
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[k] = z;
  }
  std::sort(x, x + n);
  for (int k = 0; k < n; ++k) {
    double P, dP;
    jacobi_p(n, alpha, x[k], P, dP);
    w[k] = std::pow(2.0, alpha + 1.0) / ((1.0 - x[k] * x[k]) * dP * dP);
  }
}

void tet_rule(int degree, std::vector<double>& rstw) {
  const int n = degree / 2 + 1;
  std::vector<double> a(n), wa(n), b(n), wb(n), c(n), wc(n);
  gauss_jacobi(n, 0.0, a.data(), wa.data());
  gauss_jacobi(n, 1.0, b.data(), wb.data());
  gauss_jacobi(n, 2.0, c.data(), wc.data());
  rstw.assign(size_t(n) * n * n * 4, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        double* o = &rstw[((size_t(i) * n + j) * n + k) * 4];
        o[0] = (1 + a[i]) * (1 - b[j]) * (1 - c[k]) / 4 - 1;
        o[1] = (1 + b[j]) * (1 - c[k]) / 2 - 1;
        o[2] = c[k];
        o[3] = wa[i] * wb[j] * wc[k] / 8;
      }
}

void tri_rule(int degree, std::vector<double>& uvw) {
  const int n = degree / 2 + 1;
  std::vector<double> a(n), wa(n), b(n), wb(n);
  gauss_jacobi(n, 0.0, a.data(), wa.data());
  gauss_jacobi(n, 1.0, b.data(), wb.data());
  uvw.assign(size_t(n) * n * 3, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double* o = &uvw[(size_t(i) * n + j) * 3];
      o[0] = (1 + a[i]) * (1 - b[j]) / 2 - 1;
      o[1] = b[j];
      o[2] = wa[i] * wb[j] / 2;
    }
}

bool build_modal_ops(const RefElement& re, ModalOps& out, std::string& err) {
  const int p = re.p, Np = re.Np, Nfp = re.Nfp;
  static const double kRef[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
  tet_rule(2 * p, out.vol);
  tri_rule(2 * p + 1, out.face);
  const int Nq = int(out.vol.size() / 4), Nfq = int(out.face.size() / 3);
  out.Nq = Nq;
  out.Nfq = Nfq;
  // Lagrange values at points: eval_basis(points) invV
  auto lagrange = [&](const std::vector<double>& pts, int n, std::vector<double>& L) {
    std::vector<double> r(n), s(n), t(n), psi(size_t(n) * Np);
    for (int q = 0; q < n; ++q) { r[q] = pts[3 * q]; s[q] = pts[3 * q + 1]; t[q] = pts[3 * q + 2]; }
    eval_basis(p, n, r.data(), s.data(), t.data(), psi.data());
    L.assign(size_t(n) * Np, 0.0);
    for (int q = 0; q < n; ++q)
      for (int j = 0; j < Np; ++j) {
        double acc = 0.0;
        for (int m = 0; m < Np; ++m) acc += psi[size_t(q) * Np + m] * re.invV[size_t(m) * Np + j];
        L[size_t(q) * Np + j] = acc;
      }
  };
  // M^-1 = V V^T with V = invV^-1
  std::vector<double> V = re.invV;
  if (!invert_matrix(Np, V)) { err = "singular inverse Vandermonde"; return false; }
  std::vector<double> Minv(size_t(Np) * Np, 0.0);
  for (int a = 0; a < Np; ++a)
    for (int b = 0; b < Np; ++b) {
      double acc = 0.0;
      for (int m = 0; m < Np; ++m) acc += V[size_t(a) * Np + m] * V[size_t(b) * Np + m];
      Minv[size_t(a) * Np + b] = acc;
    }
  // volume
  std::vector<double> vpts(size_t(Nq) * 3);
  for (int q = 0; q < Nq; ++q)
    for (int d = 0; d < 3; ++d) vpts[3 * q + d] = out.vol[4 * q + d];
  lagrange(vpts, Nq, out.Iq);
  const std::vector<double>* D[3] = {&re.Dr, &re.Ds, &re.Dt};
  out.Sv.assign(size_t(3) * Np * Nq, 0.0);
  std::vector<double> dl(Np, 0.0);
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < Nq; ++q) {
      for (int j = 0; j < Np; ++j) {
        double acc = 0.0;
        for (int m = 0; m < Np; ++m) acc += out.Iq[size_t(q) * Np + m] * (*D[a])[size_t(m) * Np + j];
        dl[j] = acc;
      }
      for (int n = 0; n < Np; ++n) {
        double acc = 0.0;
        for (int j = 0; j < Np; ++j) acc += Minv[size_t(n) * Np + j] * dl[j];
        out.Sv[(size_t(a) * Np + n) * Nq + q] = acc * out.vol[4 * q + 3];
      }
    }
  // faces: variant 0 = own rule, 1 + o = the neighbour's rule through orientation o
  out.Ifn.assign(size_t(4) * 7 * Nfq * Nfp, 0.0);
  out.Sf.assign(size_t(4) * 7 * Np * Nfq, 0.0);
  std::vector<double> fpts(size_t(Nfq) * 3), L;
  for (int f = 0; f < 4; ++f)
    for (int var = 0; var < 7; ++var) {
      for (int q = 0; q < Nfq; ++q) {
        const double u = out.face[3 * q], v = out.face[3 * q + 1];
        const double lam[3] = {-(u + v) / 2, (1 + u) / 2, (1 + v) / 2};
        for (int d = 0; d < 3; ++d) {
          double x = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double l = var == 0 ? lam[c] : lam[kPerm[var - 1][c]];
            x += l * kRef[kFaceVerts[f][c]][d];
          }
          fpts[3 * q + d] = x;
        }
      }
      lagrange(fpts, Nfq, L);
      const size_t fv = size_t(f) * 7 + var;
      for (int q = 0; q < Nfq; ++q)
        for (int m = 0; m < Nfp; ++m)
          out.Ifn[(fv * Nfq + q) * Nfp + m] = L[size_t(q) * Np + re.Fmask[f * Nfp + m]];
      for (int n = 0; n < Np; ++n)
        for (int q = 0; q < Nfq; ++q) {
          double acc = 0.0;
          for (int j = 0; j < Np; ++j) acc += Minv[size_t(n) * Np + j] * L[size_t(q) * Np + j];
          out.Sf[(fv * Np + n) * Nfq + q] = acc * out.face[3 * q + 2];
        }
    }
  return true;
}

}  // namespace dg
