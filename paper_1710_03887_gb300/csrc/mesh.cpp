// Mesh processing: geometric factors of the affine element maps and face
// connectivity (the partition of Appendix A, Eq. 9, and the shared faces that
// carry the numerical flux of Eq. 10).
//
// Per element, from the map x = ( -(1+r+s+t) v1 + (1+r) v2 + (1+s) v3 + (1+t) v4 ) / 2:
//   J            determinant of dx/d(r,s,t)
//   drdx[a][b]   d r_a / d x_b (inverse of the Jacobian matrix)
//   face normals from the reference-gradient identities
//     face 1 (t=-1): -grad t,  face 2 (s=-1): -grad s,
//     face 3 (r+s+t=-1): grad r + grad s + grad t,  face 4 (r=-1): -grad r;
//   sJ = |unnormalised normal| * J  (physical area per unit parameter area),
//   Fscale = sJ / J.
// Faces are matched combinatorially: the key of a face is its sorted triple of
// vertex identities (the caller may identify vertices, e.g. for periodic
// boxes). The orientation code says which of the six vertex correspondences
// maps the face onto its neighbour's.
#include <algorithm>
#include <array>
#include <cmath>
#include <unordered_map>

#include "dg_host.hpp"

namespace dg {

namespace {
struct KeyHash {
  size_t operator()(const std::array<int64_t, 3>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 3; ++i) {
      h ^= uint64_t(k[i]) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
      h *= 1099511628211ull;
    }
    return size_t(h);
  }
};
}  // namespace

bool build_mesh(const RefElement& ref, int64_t nvert, const double* xyz, int64_t K,
                const int32_t* EToV, const int8_t* face_tag, const int64_t* vclass,
                Mesh& m, std::string& err) {
  (void)ref;
  if (K <= 0 || nvert < 4 || !xyz || !EToV) { err = "empty mesh or null arrays"; return false; }
  m.K = K;
  m.verts.assign(size_t(K) * 12, 0.0);
  m.J.assign(K, 0.0);
  m.drdx.assign(size_t(K) * 9, 0.0);
  m.nrm.assign(size_t(K) * 12, 0.0);
  m.sJ.assign(size_t(K) * 4, 0.0);
  m.Fscale.assign(size_t(K) * 4, 0.0);
  m.rin.assign(K, 0.0);
  for (int64_t e = 0; e < K; ++e) {
    double v[4][3];
    for (int a = 0; a < 4; ++a) {
      const int32_t id = EToV[e * 4 + a];
      if (id < 0 || id >= nvert) { err = "EToV entry out of range at element " + std::to_string(e); return false; }
      for (int d = 0; d < 3; ++d) v[a][d] = xyz[size_t(id) * 3 + d];
      for (int d = 0; d < 3; ++d) m.verts[size_t(e) * 12 + a * 3 + d] = v[a][d];
    }
    // Jacobian matrix: column c is dx/d(r,s,t)_c
    double A[3][3];
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) A[d][c] = 0.5 * (v[c + 1][d] - v[0][d]);
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(det > 0.0)) { err = "inverted or degenerate element " + std::to_string(e); return false; }
    m.J[e] = det;
    // inverse via cofactors: drdx[a][b] = d r_a / d x_b
    double inv[3][3];
    inv[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
    inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    inv[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
    inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    inv[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
    inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) m.drdx[size_t(e) * 9 + a * 3 + b] = inv[a][b];
    double area_sum = 0.0;
    for (int f = 0; f < 4; ++f) {
      double n[3];
      for (int b = 0; b < 3; ++b) {
        switch (f) {
          case 0: n[b] = -inv[2][b]; break;
          case 1: n[b] = -inv[1][b]; break;
          case 2: n[b] = inv[0][b] + inv[1][b] + inv[2][b]; break;
          default: n[b] = -inv[0][b]; break;
        }
      }
      const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      for (int b = 0; b < 3; ++b) m.nrm[size_t(e) * 12 + f * 3 + b] = n[b] / len;
      m.sJ[size_t(e) * 4 + f] = len * det;
      m.Fscale[size_t(e) * 4 + f] = len;
      area_sum += 2.0 * len * det;
    }
    m.rin[e] = 3.0 * (det * 4.0 / 3.0) / area_sum;
  }
  // connectivity
  m.EToE.assign(size_t(K) * 4, -1);
  m.EToF.assign(size_t(K) * 4, 0);
  m.orient.assign(size_t(K) * 4, 0);
  m.bc.assign(size_t(K) * 4, -1);
  auto cls = [&](int64_t e, int a) -> int64_t {
    const int32_t id = EToV[e * 4 + a];
    return vclass ? vclass[id] : int64_t(id);
  };
  std::unordered_map<std::array<int64_t, 3>, int64_t, KeyHash> open;
  open.reserve(size_t(K) * 2);
  for (int64_t e = 0; e < K; ++e) {
    for (int f = 0; f < 4; ++f) {
      std::array<int64_t, 3> key = {cls(e, kFaceVerts[f][0]), cls(e, kFaceVerts[f][1]),
                                    cls(e, kFaceVerts[f][2])};
      std::sort(key.begin(), key.end());
      if (key[0] == key[1] || key[1] == key[2]) {
        err = "face with repeated vertices at element " + std::to_string(e);
        return false;
      }
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, e * 4 + f);
        continue;
      }
      const int64_t other = it->second;
      if (other < 0) { err = "non-manifold face at element " + std::to_string(e); return false; }
      const int64_t e2 = other / 4;
      const int f2 = int(other % 4);
      it->second = -1;   // closed; a third hit is an error
      int o1 = -1, o2 = -1;
      for (int o = 0; o < 6; ++o) {
        bool ok1 = true, ok2 = true;
        for (int c = 0; c < 3; ++c) {
          ok1 = ok1 && cls(e, kFaceVerts[f][c]) == cls(e2, kFaceVerts[f2][kPerm[o][c]]);
          ok2 = ok2 && cls(e2, kFaceVerts[f2][c]) == cls(e, kFaceVerts[f][kPerm[o][c]]);
        }
        if (ok1 && o1 < 0) o1 = o;
        if (ok2 && o2 < 0) o2 = o;
      }
      if (o1 < 0 || o2 < 0) { err = "face orientation not found"; return false; }
      double dot = 0.0;
      for (int b = 0; b < 3; ++b)
        dot += m.nrm[size_t(e) * 12 + f * 3 + b] * m.nrm[size_t(e2) * 12 + f2 * 3 + b];
      if (dot > -1.0 + 1e-8) {
        err = "matched faces are not back to back at element " + std::to_string(e);
        return false;
      }
      m.EToE[e * 4 + f] = int32_t(e2);
      m.EToF[e * 4 + f] = int8_t(f2);
      m.orient[e * 4 + f] = int8_t(o1);
      m.EToE[e2 * 4 + f2] = int32_t(e);
      m.EToF[e2 * 4 + f2] = int8_t(f);
      m.orient[e2 * 4 + f2] = int8_t(o2);
    }
  }
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 4; ++f) {
      const int8_t tag = face_tag ? face_tag[e * 4 + f] : int8_t(0);
      if (m.EToE[e * 4 + f] < 0) {
        if (tag < 0) { err = "untagged boundary face at element " + std::to_string(e); return false; }
        if (tag >= 8) { err = "boundary id must be < 8"; return false; }
        m.bc[e * 4 + f] = tag;
        m.EToE[e * 4 + f] = -1;
      }
    }
  return true;
}

}  // namespace dg
