// Host-side data of the DG Euler library: reference-element operators and
// processed mesh. Everything here is plain C++ (no CUDA) and float64.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace dg {

constexpr int kMaxOrder = 4;

inline int num_nodes(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
inline int num_face_nodes(int p) { return (p + 1) * (p + 2) / 2; }

// Reference tetrahedron with vertices v1=(-1,-1,-1), v2=(1,-1,-1), v3=(-1,1,-1),
// v4=(-1,-1,1); faces 1: t=-1, 2: s=-1, 3: r+s+t=-1, 4: r=-1.
struct RefElement {
  int p = 0, Np = 0, Nfp = 0;
  std::vector<double> r, s, t;            // node coordinates [Np]
  std::vector<int> lat;                   // lattice index (i,j,k) per node [Np*3]
  std::vector<double> Dr, Ds, Dt;         // [Np*Np], row-major (i, j)
  std::vector<double> LIFT;               // [Np * 4Nfp], row-major
  std::vector<double> face_w;             // [4*Nfp] column sums of the face mass
  std::vector<int> Fmask;                 // [4*Nfp] volume node of face node
  std::vector<double> invV;               // [Np*Np] inverse Vandermonde (modal coefficients)
  // neighbour face-node table: node of the neighbour matching own face node m,
  // indexed ((f*4 + f2)*6 + perm)*Nfp + m
  std::vector<uint8_t> nbr_node;
};

// Canonical vertex triple of each reference face (0-based local vertex ids)
extern const int kFaceVerts[4][3];
// The six permutations of a face's vertex triple, in the order used for the
// orientation code: own face vertex i matches neighbour face vertex kPerm[o][i]
extern const int kPerm[6][3];

bool build_ref_element(int p, RefElement& out, std::string& err);
// Orthonormal basis values at arbitrary reference points: out[npts * Np]
void eval_basis(int p, int npts, const double* r, const double* s, const double* t,
                double* out);

// Processed mesh (element order as uploaded)
struct Mesh {
  int64_t K = 0;
  std::vector<double> verts;              // [K*4*3] vertex coordinates per element
  std::vector<double> J;                  // [K]
  std::vector<double> drdx;               // [K*9]: d r_a / d x_b at a*3+b
  std::vector<double> nrm;                // [K*4*3] outward unit normals
  std::vector<double> sJ;                 // [K*4] face area / 2
  std::vector<double> Fscale;             // [K*4] sJ / J
  std::vector<int32_t> EToE;              // [K*4] neighbour element, or -1 on a boundary
  std::vector<int8_t> EToF;               // [K*4] neighbour face (0..3)
  std::vector<int8_t> orient;             // [K*4] orientation code (0..5)
  std::vector<int8_t> bc;                 // [K*4] boundary id, -1 on interior faces
  std::vector<double> rin;                // [K] inscribed radius 3V / sum(face areas)
};

// Geometric factors and face matching. ``face_tag`` (nullable): boundary id
// (0..7) of each face; read only on faces without a neighbour, where a
// negative tag is an error. NULL gives id 0 to every boundary face. ``vclass`` (nullable):
// connectivity identity of each vertex (periodic identification).
bool build_mesh(const RefElement& ref, int64_t nvert, const double* xyz, int64_t K,
                const int32_t* EToV, const int8_t* face_tag, const int64_t* vclass,
                Mesh& out, std::string& err);

bool invert_matrix(int n, std::vector<double>& a);   // in place, row-major

// The paper's discretisation (modal_ops.cpp): Gauss rules and the operators
// of the weak form on nodal values (see there for the formulas).
struct ModalOps {
  int Nq = 0, Nfq = 0;
  std::vector<double> vol;                // [Nq][4]: r, s, t, weight (degree 2p)
  std::vector<double> face;               // [Nfq][3]: u, v, weight (degree 2p + 1)
  std::vector<double> Iq;                 // [Nq][Np] Lagrange basis at the volume points
  std::vector<double> Sv;                 // [3][Np][Nq] volume weights of G_r, G_s, G_t
  std::vector<double> Ifn;                // [4][7][Nfq][Nfp] face nodes -> face points
  std::vector<double> Sf;                 // [4][7][Np][Nfq] surface weights of F*
};
// n-point Gauss rule for the weight (1 - x)^alpha on [-1, 1]
void gauss_jacobi(int n, double alpha, double* x, double* w);
void tet_rule(int degree, std::vector<double>& rstw);
void tri_rule(int degree, std::vector<double>& uvw);
bool build_modal_ops(const RefElement& re, ModalOps& out, std::string& err);

}  // namespace dg
