// Reference-element operators of the nodal DG method.
//
// The paper expands the solution on each element in an L2-orthonormal
// polynomial basis of degree p (Appendix A, Eq. 11), which makes the modal
// mass matrix the identity. The library keeps nodal unknowns but builds
// every operator from that orthonormal basis (the Proriol-Koornwinder-Dubiner
// product of normalised Jacobi polynomials on the collapsed cube):
//   V[i][m]   = psi_m(x_i)                   (Vandermonde)
//   D_r       = V_r V^-1                      (derivative of the interpolant)
//   M^-1      = V V^T                         (orthonormality)
//   E_f       = face mass matrix (V_f V_f^T)^-1 in the face's parameters
//   LIFT      = M^-1 [E_1 E_2 E_3 E_4]
// Nodes are Warburton's warp-and-blend points with blending exponent zero:
// equispaced lattice points moved so that each edge carries the 1D
// Legendre-Gauss-Lobatto points, the edge displacement being blended into
// faces and the interior.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dg_host.hpp"

namespace dg {

const int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// ------------------------------------------------------------------ algebra

bool invert_matrix(int n, std::vector<double>& a) {
  std::vector<double> inv(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) inv[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[size_t(r) * n + c]) > std::fabs(a[size_t(piv) * n + c])) piv = r;
    if (std::fabs(a[size_t(piv) * n + c]) < 1e-300) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[size_t(piv) * n + k], a[size_t(c) * n + k]);
        std::swap(inv[size_t(piv) * n + k], inv[size_t(c) * n + k]);
      }
    const double d = 1.0 / a[size_t(c) * n + c];
    for (int k = 0; k < n; ++k) {
      a[size_t(c) * n + k] *= d;
      inv[size_t(c) * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[size_t(r) * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[size_t(r) * n + k] -= f * a[size_t(c) * n + k];
        inv[size_t(r) * n + k] -= f * inv[size_t(c) * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

static void matmul(int n, int k, int m, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double acc = 0.0;
      for (int l = 0; l < k; ++l) acc += A[size_t(i) * k + l] * B[size_t(l) * m + j];
      C[size_t(i) * m + j] = acc;
    }
}

// ------------------------------------------------------- 1D building blocks

// Legendre P_n and P_n' at x by the three-term recurrence.
static void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    const double d2 = d0 + (2 * k + 1) * p1;   // P'_{k+1} = P'_{k-1} + (2k+1) P_k
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  P = p1; dP = d1;
}

// Legendre-Gauss-Lobatto points: -1, 1 and the zeros of P_p', by Newton from
// the Chebyshev-Lobatto points.
static std::vector<double> lgl(int p) {
  std::vector<double> x(p + 1);
  x[0] = -1.0; x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double z = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, z, P, dP);
      // P'' from the Legendre equation (1-z^2) P'' = 2 z P' - p(p+1) P
      const double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
      const double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  std::sort(x.begin(), x.end());
  return x;
}

// phi(x) = w(x) / (1 - x^2) where w interpolates, on the p+1 equispaced points
// of [-1,1], the displacement from each equispaced point to its LGL point.
static double warp_over_bubble(int p, const std::vector<double>& disp, double x) {
  double phi = 0.0;
  for (int i = 1; i < p; ++i) {
    const double xi = -1.0 + 2.0 * i / p;
    double term = disp[i] / (1.0 - xi * xi);
    for (int j = 1; j < p; ++j) {
      if (j == i) continue;
      const double xj = -1.0 + 2.0 * j / p;
      term *= (x - xj) / (xi - xj);
    }
    phi += term;
  }
  return phi;
}

// Normalised Jacobi polynomial P_n^{(a,b)}(x): orthonormal for the weight
// (1-x)^a (1+x)^b on [-1,1]; three-term recurrence.
static double jacobi(int n, double a, double b, double x) {
  const double g0 = std::pow(2.0, a + b + 1.0) / (a + b + 1.0) * std::tgamma(a + 1.0) *
                    std::tgamma(b + 1.0) / std::tgamma(a + b + 1.0);
  double pm = 1.0 / std::sqrt(g0);
  if (n == 0) return pm;
  const double g1 = (a + 1.0) * (b + 1.0) / (a + b + 3.0) * g0;
  double pc = ((a + b + 2.0) * x / 2.0 + (a - b) / 2.0) / std::sqrt(g1);
  if (n == 1) return pc;
  double aold = 2.0 / (2.0 + a + b) * std::sqrt((a + 1.0) * (b + 1.0) / (a + b + 3.0));
  for (int i = 1; i < n; ++i) {
    const double h1 = 2.0 * i + a + b;
    const double anew = 2.0 / (h1 + 2.0) *
        std::sqrt((i + 1.0) * (i + 1.0 + a + b) * (i + 1.0 + a) * (i + 1.0 + b) /
                  (h1 + 1.0) / (h1 + 3.0));
    const double bnew = -(a * a - b * b) / h1 / (h1 + 2.0);
    const double pn = (-aold * pm + (x - bnew) * pc) / anew;
    pm = pc; pc = pn; aold = anew;
  }
  return pc;
}

// d/dx of the normalised Jacobi polynomial
static double djacobi(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + a + b + 1.0)) * jacobi(n - 1, a + 1.0, b + 1.0, x);
}

static double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// Collapsed coordinates of the tetrahedron
static void collapse3(double r, double s, double t, double& a, double& b, double& c) {
  a = (std::fabs(s + t) > 1e-14) ? 2.0 * (1.0 + r) / (-s - t) - 1.0 : -1.0;
  b = (std::fabs(t - 1.0) > 1e-14) ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0 : -1.0;
  c = t;
}

// Orthonormal tetrahedral mode (i,j,k) and, optionally, its gradient:
//   psi = 2 sqrt(2) P_i(a) P_j^(2i+1,0)(b) (1-b)^i P_k^(2i+2j+2,0)(c) (1-c)^(i+j)
// with normalised Jacobi polynomials; in the collapsed coordinates
// dr ds dt = (1-b)(1-c)^2/8 da db dc, which makes the modes orthonormal.
static void mode3(int i, int j, int k, double r, double s, double t, double* val,
                  double* dr, double* ds, double* dt) {
  double a, b, c;
  collapse3(r, s, t, a, b, c);
  const double A = jacobi(i, 0, 0, a), dA = djacobi(i, 0, 0, a);
  const double B = jacobi(j, 2 * i + 1, 0, b), dB = djacobi(j, 2 * i + 1, 0, b);
  const double C = jacobi(k, 2 * (i + j) + 2, 0, c), dC = djacobi(k, 2 * (i + j) + 2, 0, c);
  const double hb = 1.0 - b, hc = 1.0 - c;
  const double norm = 2.0 * std::sqrt(2.0);
  if (val) *val = norm * A * B * ipow(hb, i) * C * ipow(hc, i + j);
  if (!dr) return;
  // chain rule through a(r,s,t), b(s,t), c(t):
  //   da/dr = 4/(hb hc),  da/ds = da/dt = 2(1+a)/(hb hc),
  //   db/ds = 2/hc,       db/dt = (1+b)/hc,        dc/dt = 1.
  // Each power of hb, hc that a derivative divides out is taken from the
  // factor it multiplies, so nothing is singular at the collapsed edges.
  const double fa = (i >= 1) ? 4.0 * dA * B * ipow(hb, i - 1) * C * ipow(hc, i + j - 1) : 0.0;
  double gb = dB * ipow(hb, i);                  // d/db of B(b) hb^i
  if (i >= 1) gb -= i * B * ipow(hb, i - 1);
  const double fb = (i + j >= 1) ? 2.0 * A * gb * C * ipow(hc, i + j - 1) : 0.0;
  double gc = dC * ipow(hc, i + j);              // d/dc of C(c) hc^(i+j)
  if (i + j >= 1) gc -= (i + j) * C * ipow(hc, i + j - 1);
  const double fc = A * B * ipow(hb, i) * gc;
  *dr = norm * fa;
  *ds = norm * (0.5 * (1.0 + a) * fa + fb);
  *dt = norm * (0.5 * (1.0 + a) * fa + 0.5 * (1.0 + b) * fb + fc);
}

// Orthonormal triangle mode (i,j) on u,v >= -1, u+v <= 0:
//   sqrt(2) P_i(a) P_j^(2i+1,0)(b) (1-b)^i,  du dv = (1-b)/2 da db
static double mode2(int i, int j, double u, double v) {
  const double a = (std::fabs(v - 1.0) > 1e-14) ? 2.0 * (1.0 + u) / (1.0 - v) - 1.0 : -1.0;
  const double b = v;
  return std::sqrt(2.0) * jacobi(i, 0, 0, a) * jacobi(j, 2 * i + 1, 0, b) * ipow(1.0 - b, i);
}

void eval_basis(int p, int npts, const double* r, const double* s, const double* t,
                double* out) {
  const int Np = num_nodes(p);
  for (int q = 0; q < npts; ++q) {
    int m = 0;
    for (int i = 0; i <= p; ++i)
      for (int j = 0; j <= p - i; ++j)
        for (int k = 0; k <= p - i - j; ++k) {
          mode3(i, j, k, r[q], s[q], t[q], &out[size_t(q) * Np + m], nullptr, nullptr, nullptr);
          ++m;
        }
  }
}

// ------------------------------------------------------------------- nodes

static void warp_blend_nodes(int p, RefElement& re) {
  const int Np = num_nodes(p);
  re.r.assign(Np, 0); re.s.assign(Np, 0); re.t.assign(Np, 0); re.lat.assign(3 * Np, 0);
  const double s3 = std::sqrt(3.0), s6 = std::sqrt(6.0);
  const double X[4][3] = {{-1.0, -1.0 / s3, -1.0 / s6}, {1.0, -1.0 / s3, -1.0 / s6},
                          {0.0, 2.0 / s3, -1.0 / s6}, {0.0, 0.0, 3.0 / s6}};
  const std::vector<double> xg = lgl(p);
  std::vector<double> disp(p + 1);
  for (int i = 0; i <= p; ++i) disp[i] = xg[i] - (-1.0 + 2.0 * i / p);
  const int opp[4] = {3, 2, 0, 1};
  const double tol = 1e-10;
  int n = 0;
  for (int k = 0; k <= p; ++k)
    for (int j = 0; j <= p - k; ++j)
      for (int i = 0; i <= p - k - j; ++i, ++n) {
        re.lat[3 * n] = i; re.lat[3 * n + 1] = j; re.lat[3 * n + 2] = k;
        const double L[4] = {double(p - i - j - k) / p, double(i) / p, double(j) / p,
                             double(k) / p};
        double pos[3] = {0, 0, 0};
        for (int v = 0; v < 4; ++v)
          for (int d = 0; d < 3; ++d) pos[d] += L[v] * X[v][d];
        int nzero = 0;
        for (int v = 0; v < 4; ++v) nzero += (L[v] < tol);
        double shift[3] = {0, 0, 0};
        for (int f = 0; f < 4; ++f) {
          const int* fv = kFaceVerts[f];
          const int o = opp[f];
          double warp[3] = {0, 0, 0};
          for (int e = 0; e < 3; ++e) {
            const int u = fv[e], w = fv[(e + 1) % 3];
            const double amt = 4.0 * L[u] * L[w] * warp_over_bubble(p, disp, L[w] - L[u]);
            for (int d = 0; d < 3; ++d) warp[d] += amt * 0.5 * (X[w][d] - X[u][d]);
          }
          const double den = (L[fv[0]] + 0.5 * L[o]) * (L[fv[1]] + 0.5 * L[o]) *
                             (L[fv[2]] + 0.5 * L[o]);
          const double blend = den > tol ? L[fv[0]] * L[fv[1]] * L[fv[2]] / den : 0.0;
          for (int d = 0; d < 3; ++d) shift[d] += blend * warp[d];
          if (nzero == 2 && L[o] < tol)
            for (int d = 0; d < 3; ++d) shift[d] = warp[d];
        }
        for (int d = 0; d < 3; ++d) pos[d] += shift[d];
        // barycentrics of the warped point in the equilateral tetrahedron
        double A[9], rhs[3];
        for (int d = 0; d < 3; ++d) {
          A[d * 3 + 0] = X[1][d] - X[0][d];
          A[d * 3 + 1] = X[2][d] - X[0][d];
          A[d * 3 + 2] = X[3][d] - X[0][d];
          rhs[d] = pos[d] - X[0][d];
        }
        std::vector<double> Ai(A, A + 9);
        invert_matrix(3, Ai);
        double mu[3];
        for (int a = 0; a < 3; ++a)
          mu[a] = Ai[a * 3] * rhs[0] + Ai[a * 3 + 1] * rhs[1] + Ai[a * 3 + 2] * rhs[2];
        re.r[n] = -1.0 + 2.0 * mu[0];
        re.s[n] = -1.0 + 2.0 * mu[1];
        re.t[n] = -1.0 + 2.0 * mu[2];
      }
}

// --------------------------------------------------------------- operators

bool build_ref_element(int p, RefElement& re, std::string& err) {
  if (p < 1 || p > kMaxOrder) {
    err = "order must be between 1 and " + std::to_string(kMaxOrder);
    return false;
  }
  re.p = p;
  const int Np = num_nodes(p), Nfp = num_face_nodes(p);
  re.Np = Np; re.Nfp = Nfp;
  warp_blend_nodes(p, re);
  std::vector<double> V(size_t(Np) * Np), Vr(V.size()), Vs(V.size()), Vt(V.size());
  for (int n = 0; n < Np; ++n) {
    int m = 0;
    for (int i = 0; i <= p; ++i)
      for (int j = 0; j <= p - i; ++j)
        for (int k = 0; k <= p - i - j; ++k, ++m)
          mode3(i, j, k, re.r[n], re.s[n], re.t[n], &V[size_t(n) * Np + m],
                &Vr[size_t(n) * Np + m], &Vs[size_t(n) * Np + m], &Vt[size_t(n) * Np + m]);
  }
  std::vector<double> Vi = V;
  if (!invert_matrix(Np, Vi)) { err = "singular Vandermonde"; return false; }
  re.invV = Vi;
  re.Dr.assign(size_t(Np) * Np, 0); re.Ds = re.Dr; re.Dt = re.Dr;
  matmul(Np, Np, Np, Vr.data(), Vi.data(), re.Dr.data());
  matmul(Np, Np, Np, Vs.data(), Vi.data(), re.Ds.data());
  matmul(Np, Np, Np, Vt.data(), Vi.data(), re.Dt.data());
  // face node lists (increasing volume node order)
  re.Fmask.assign(4 * Nfp, -1);
  for (int f = 0; f < 4; ++f) {
    int m = 0;
    for (int n = 0; n < Np; ++n) {
      const int i = re.lat[3 * n], j = re.lat[3 * n + 1], k = re.lat[3 * n + 2];
      const bool on = (f == 0 && k == 0) || (f == 1 && j == 0) || (f == 2 && i + j + k == p) ||
                      (f == 3 && i == 0);
      if (on) re.Fmask[f * Nfp + m++] = n;
    }
    if (m != Nfp) { err = "face node count mismatch"; return false; }
  }
  // face mass matrices in the face parameters (r,s), (r,t), (s,t), (s,t)
  std::vector<double> Emat(size_t(Np) * 4 * Nfp, 0.0);
  re.face_w.assign(4 * Nfp, 0.0);
  for (int f = 0; f < 4; ++f) {
    std::vector<double> V2(size_t(Nfp) * Nfp);
    for (int m = 0; m < Nfp; ++m) {
      const int n = re.Fmask[f * Nfp + m];
      const double u = (f <= 1) ? re.r[n] : re.s[n];
      const double v = (f == 0) ? re.s[n] : re.t[n];
      int q = 0;
      for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p - i; ++j, ++q) V2[size_t(m) * Nfp + q] = mode2(i, j, u, v);
    }
    std::vector<double> MM(size_t(Nfp) * Nfp, 0.0);   // V2 V2^T, then inverted
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b) {
        double acc = 0;
        for (int q = 0; q < Nfp; ++q) acc += V2[size_t(a) * Nfp + q] * V2[size_t(b) * Nfp + q];
        MM[size_t(a) * Nfp + b] = acc;
      }
    if (!invert_matrix(Nfp, MM)) { err = "singular face Vandermonde"; return false; }
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b) {
        Emat[size_t(re.Fmask[f * Nfp + a]) * 4 * Nfp + f * Nfp + b] = MM[size_t(a) * Nfp + b];
        re.face_w[f * Nfp + b] += MM[size_t(a) * Nfp + b];
      }
  }
  // LIFT = V V^T E
  std::vector<double> VVt(size_t(Np) * Np);
  for (int a = 0; a < Np; ++a)
    for (int b = 0; b < Np; ++b) {
      double acc = 0;
      for (int q = 0; q < Np; ++q) acc += V[size_t(a) * Np + q] * V[size_t(b) * Np + q];
      VVt[size_t(a) * Np + b] = acc;
    }
  re.LIFT.assign(size_t(Np) * 4 * Nfp, 0.0);
  matmul(Np, Np, 4 * Nfp, VVt.data(), Emat.data(), re.LIFT.data());
  // neighbour face-node table from the node lattice: a face node is fixed by
  // its barycentric weights on the face's three vertices
  re.nbr_node.assign(size_t(4) * 4 * 6 * Nfp, 0xFF);
  auto bary = [&](int n, int v) {
    const int i = re.lat[3 * n], j = re.lat[3 * n + 1], k = re.lat[3 * n + 2];
    const int L[4] = {p - i - j - k, i, j, k};
    return L[v];
  };
  for (int f = 0; f < 4; ++f)
    for (int f2 = 0; f2 < 4; ++f2)
      for (int o = 0; o < 6; ++o)
        for (int m = 0; m < Nfp; ++m) {
          const int n = re.Fmask[f * Nfp + m];
          int found = -1;
          for (int m2 = 0; m2 < Nfp; ++m2) {
            const int n2 = re.Fmask[f2 * Nfp + m2];
            bool ok = true;
            for (int c = 0; c < 3; ++c)
              ok = ok && bary(n, kFaceVerts[f][c]) == bary(n2, kFaceVerts[f2][kPerm[o][c]]);
            if (ok) { found = n2; break; }
          }
          if (found < 0) { err = "face node table incomplete"; return false; }
          re.nbr_node[((size_t(f) * 4 + f2) * 6 + o) * Nfp + m] = uint8_t(found);
        }
  return true;
}

}  // namespace dg
