// C ABI of the DG Euler library (declared in include/dg_euler.h): context,
// mesh upload, device buffers and the time-stepping loop.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dg_euler.h"
#include "dg_device.cuh"
#include "dg_host.hpp"
#include "ghost_f32.cuh"

namespace {

// Carpenter & Kennedy (1994), five-stage 2N-storage fourth-order Runge-Kutta
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0,
                        -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0,
                        -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};
const double kRkC[5] = {0.0, 1432997174477.0 / 9575080441755.0,
                        2526269341429.0 / 6820363962896.0, 2006345519317.0 / 3224310063776.0,
                        2802321613138.0 / 2924317926251.0};

// Heun's method (the paper's second-order Runge-Kutta, section 1.1) in the
// same 2N-storage form: res = dt f(q); q1 = q + res; res = -res + dt f(q1);
// q2 = q1 + res/2 = (q + q1 + dt f(q1))/2.
const double kHeunA[2] = {0.0, -1.0};
const double kHeunB[2] = {1.0, 0.5};
const double kHeunC[2] = {0.0, 1.0};

constexpr int kTotalsBlocks = 256;

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Face-node tables [4][4][6][Nfp], one after the other, indexed by (own face
// f, neighbour face f2, orientation code o, own face node m): the
// neighbour's volume node at the same point, then that node's index in the
// neighbour face's node list. Uploaded for the stage kernels and read back
// by dg_face_pairs.
std::vector<uint8_t> face_node_tables(const dg::RefElement& re) {
  const int Nfp = re.Nfp;
  std::vector<uint8_t> t(re.nbr_node);
  t.resize(2 * re.nbr_node.size(), 0xFF);
  for (int f = 0; f < 4; ++f)
    for (int f2 = 0; f2 < 4; ++f2)
      for (int o = 0; o < 6; ++o)
        for (int m = 0; m < Nfp; ++m) {
          const size_t i = ((size_t(f) * 4 + f2) * 6 + o) * Nfp + m;
          for (int m2 = 0; m2 < Nfp; ++m2)
            if (re.Fmask[f2 * Nfp + m2] == re.nbr_node[i]) t[re.nbr_node.size() + i] = uint8_t(m2);
        }
  return t;
}

}  // namespace

struct dg_ctx {
  dg::RefElement ref;
  dg::Mesh mesh;
  dg_params prm{};
  int bc_mode[8];
  double inflow_amp = 0.05, inflow_alpha = 565.0;   // mouthpiece pulse (section 2.4)
  std::string err;
  cudaStream_t stream = nullptr;
  bool have_mesh = false, dev_ready = false, have_state = false;
  double t = 0.0;
  int cur = 0;
  int ntiles = 0, grid = 0, sms = 0;
  dgk::Gas gas{};
  // device buffers
  int prec = DG_PREC_FP64;
  double* q[2] = {nullptr, nullptr};
  double* res = nullptr;
  double* scratch = nullptr;       // state-sized float64: dg_eval_rhs output / staging
  // float32 perturbation form
  float* q32[2] = {nullptr, nullptr};
  float* res32 = nullptr;
  float* scratch32 = nullptr;
  float* geo32 = nullptr;
  float* ops32 = nullptr;
  double* geo = nullptr;
  int32_t* conn = nullptr;
  double* ops = nullptr;
  double* mops = nullptr;          // operators of the paper's discretisation (DG_PREC_MODAL)
  uint8_t* tbl = nullptr;
  int32_t* fmask = nullptr;
  double* ledger_part = nullptr;   // [grid][5] per-CTA ledger sums
  unsigned long long* ticket = nullptr;
  double* ledger = nullptr;        // L[5], Lres[5]
  double* mass_w = nullptr;
  double* totals_part = nullptr;   // [kTotalsBlocks*5 + 5]
  int* status = nullptr;
  // sensors
  int nprobe = 0, pcap = 0;
  int64_t precorded = 0;
  int32_t* pelem = nullptr;
  double* prow = nullptr;
  double* pring = nullptr;
  std::vector<double> mass_w_host;
  // learned closure
  float* bxyz = nullptr;           // boundary face node positions [slot][Nfp][3]
  int32_t* bface = nullptr;        // e * 4 + f of every boundary face, slot order
  int64_t nbf = 0;
  float* bpsi = nullptr;           // memory of the boundary face nodes [slot][Nfp]
  float* bpsi_res = nullptr;
  float* bD = nullptr;             // incoming-invariant increments [slot][Nfp]
  uint8_t* face_list = nullptr;    // float32 stage: faces each tile evaluates
  float* mlp_w = nullptr;          // network parameters (device), null until set
  unsigned char* mlp_img = nullptr; // their operand image for the closure kernel
  bool mlp_img_ok = false;          // image built from the current parameters
  float* mlp_m = nullptr;          // Adam moments
  float* mlp_v = nullptr;
  float* mlp_grad = nullptr;
  double* mlp_loss = nullptr;
  float* mlp_part = nullptr;       // per-block partial gradients
  size_t mlp_part_len = 0;
  int mlp_t = 0;
  double mlp_radius = 1.0;
  int64_t ntrace = 0;
  int32_t* tr_elem = nullptr;
  int8_t* tr_face = nullptr;
  float* txyz = nullptr;
  float* tr_psi = nullptr;         // memory of the trace face nodes [n][Nfp]
  float* tr_res = nullptr;
  // partitioned mesh: elements [K_own, K) are halo copies of a neighbour
  // rank's elements (not advanced; read through their cut-face nodes)
  int64_t K_own = -1;
  int64_t n_send = 0, n_recv = 0;
  int32_t* halo_send = nullptr;    // e * 4 + f of own cut faces, send order
  int32_t* halo_recv = nullptr;    // e * 4 + f of halo faces, receive order
  int stage_k = 0;                 // next Runge-Kutta stage of the step in progress
  // stage-kernel timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;   // created lazily, reused
  size_t ev_used = 0;
  void clear_events() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    ev_used = 0;
  }

  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return DG_ERR_CUDA;
  }
  void free_device() {
    if (dev_ready) cudaStreamSynchronize(stream);
    clear_events();
    dfree(q[0]); dfree(q[1]); dfree(res); dfree(scratch); dfree(geo); dfree(conn);
    dfree(ops); dfree(mops); dfree(tbl); dfree(fmask); dfree(ticket); dfree(ledger_part); dfree(ledger);
    dfree(mass_w); dfree(totals_part); dfree(status); dfree(pelem); dfree(prow); dfree(pring);
    dfree(q32[0]); dfree(q32[1]); dfree(res32); dfree(scratch32); dfree(geo32); dfree(ops32);
    dfree(bxyz); dfree(bface); dfree(bpsi); dfree(bpsi_res); dfree(bD); dfree(face_list);
    dfree(tr_elem); dfree(tr_face); dfree(txyz); dfree(tr_psi); dfree(tr_res);
    dfree(halo_send); dfree(halo_recv);
    n_send = n_recv = 0;
    ntrace = 0;
    nbf = 0;
    dev_ready = false;
    have_state = false;
    nprobe = 0;
  }
  size_t state_elems() const { return size_t(mesh.K) * 5 * ref.Np; }
  int64_t owned() const { return K_own < 0 ? mesh.K : K_own; }
  bool f32() const { return prec == DG_PREC_F32 || tc(); }
  bool tc() const { return prec == DG_PREC_F32_TC || prec == DG_PREC_F32_TC1; }
  int tc_images() const { return prec == DG_PREC_F32_TC1 ? 1 : 2; }
};

namespace {

#define DG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return c->cuda_fail(e_, #call); \
  } while (0)

// Physical position of volume node n of element e (affine map of the vertices).
void node_position(const dg_ctx* c, int64_t e, int n, double x[3]) {
  const double* v = &c->mesh.verts[size_t(e) * 12];
  const double r = c->ref.r[n], s = c->ref.s[n], t = c->ref.t[n];
  const double w[4] = {-0.5 * (1 + r + s + t), 0.5 * (1 + r), 0.5 * (1 + s), 0.5 * (1 + t)};
  for (int d = 0; d < 3; ++d) x[d] = w[0] * v[d] + w[1] * v[3 + d] + w[2] * v[6 + d] + w[3] * v[9 + d];
}

dgk::mlp::Scales mlp_scales(const dg_ctx* c) {
  return dgk::mlp::Scales{float(c->gas.rho0), float(c->gas.c0), float(c->gas.p0), float(c->gas.gm1),
                          float(1.0 / c->mlp_radius), float(1e-3 * c->mlp_radius)};
}

// Allocate and fill the device copies of the mesh and operators.
int ensure_device(dg_ctx* c) {
  if (c->dev_ready) return DG_OK;
  if (!c->have_mesh) return c->fail(DG_ERR_ORDER, "no mesh uploaded");
  const int p = c->ref.p, Np = c->ref.Np, Nfp = c->ref.Nfp, NF = 4 * Nfp;
  const int64_t K = c->mesh.K;
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
  const bool f32 = c->f32();
  const bool tcf = c->tc();
  const bool modal = c->prec == DG_PREC_MODAL;
  int bps = 0;
  if (tcf)
    DG_CUDA(dgk::stage_tc_prepare(p, c->tc_images(), &bps));
  else if (f32)
    DG_CUDA(dgk::stage_f32_prepare(p, &bps));
  else if (modal)
    DG_CUDA(dgk::stage_modal_prepare(p, &bps));
  else
    DG_CUDA(dgk::stage_prepare(p, &bps));
  if (bps < 1) return c->fail(DG_ERR_CUDA, "stage kernel does not fit on an SM");
  if (f32) DG_CUDA(dgk::closure_prepare());
  const int ET = tcf ? dgk::stage_tc_tile_elems(p)
                     : (f32 ? dgk::stage_f32_tile_elems(p)
                            : (modal ? dgk::stage_modal_tile_elems(p) : dgk::stage_tile_elems(p)));
  const int64_t Kown = c->owned();
  c->ntiles = int((Kown + ET - 1) / ET);
  // the tensor-core stage is sized for two CTAs per SM at p <= 3 (104 KB of
  // shared memory each at p = 3) and one at p = 4; a grid of that many per
  // SM is correct whatever the occupancy query says (CTAs loop over tiles)
  if (tcf) bps = std::max(bps, dgk::stage_tc_ctas_per_sm(p));
  c->grid = std::min(c->ntiles, c->sms * bps);
  const size_t nq = c->state_elems();
  if (f32) {
    DG_CUDA(cudaMalloc(&c->q32[0], nq * 4));
    DG_CUDA(cudaMalloc(&c->q32[1], nq * 4));
    DG_CUDA(cudaMalloc(&c->res32, nq * 4));
    DG_CUDA(cudaMalloc(&c->scratch32, nq * 4));
  } else {
    DG_CUDA(cudaMalloc(&c->q[0], nq * 8));
    DG_CUDA(cudaMalloc(&c->q[1], nq * 8));
    DG_CUDA(cudaMalloc(&c->res, nq * 8));
  }
  DG_CUDA(cudaMalloc(&c->scratch, nq * 8));
  // geometry records
  std::vector<double> geo(size_t(K) * dgk::kGeoStride, 0.0);
  for (int64_t e = 0; e < K; ++e) {
    double* g = &geo[size_t(e) * dgk::kGeoStride];
    for (int i = 0; i < 9; ++i) g[dgk::kGeoDrdx + i] = c->mesh.drdx[size_t(e) * 9 + i];
    for (int i = 0; i < 12; ++i) g[dgk::kGeoNrm + i] = c->mesh.nrm[size_t(e) * 12 + i];
    for (int f = 0; f < 4; ++f) {
      g[dgk::kGeoFscale + f] = c->mesh.Fscale[size_t(e) * 4 + f];
      g[dgk::kGeoSJ + f] = c->mesh.sJ[size_t(e) * 4 + f];
    }
    g[dgk::kGeoJ] = c->mesh.J[e];
  }
  DG_CUDA(cudaMalloc(&c->geo, geo.size() * 8));
  DG_CUDA(cudaMemcpy(c->geo, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice));
  if (f32) {
    std::vector<float> g32(geo.begin(), geo.end());
    DG_CUDA(cudaMalloc(&c->geo32, g32.size() * 4));
    DG_CUDA(cudaMemcpy(c->geo32, g32.data(), g32.size() * 4, cudaMemcpyHostToDevice));
  }
  // face connection words; boundary faces get a slot (their index in bfaces)
  std::vector<int32_t> conn(size_t(K) * 4);
  std::vector<int64_t> bfaces;
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 4; ++f) {
      const size_t i = size_t(e) * 4 + f;
      if (c->mesh.EToE[i] >= 0) {
        conn[i] = dgk::conn_interior(c->mesh.EToE[i], c->mesh.EToF[i], c->mesh.orient[i]);
      } else {
        // boundary id in the low 3 bits, boundary-face slot above them
        conn[i] = -1 - (c->mesh.bc[i] + 8 * int32_t(bfaces.size()));
        bfaces.push_back(int64_t(i));
      }
    }
  // node positions of every boundary face (features of the learned closure)
  if (f32 && !bfaces.empty()) {
    std::vector<float> bx(bfaces.size() * size_t(Nfp) * 3);
    for (size_t b = 0; b < bfaces.size() && !c->mesh.verts.empty(); ++b) {
      const int64_t e = bfaces[b] / 4;
      const int f = int(bfaces[b] % 4);
      for (int m = 0; m < Nfp; ++m) {
        double x[3];
        node_position(c, e, c->ref.Fmask[f * Nfp + m], x);
        for (int d = 0; d < 3; ++d) bx[(b * Nfp + m) * 3 + d] = float(x[d]);
      }
    }
    DG_CUDA(cudaMalloc(&c->bxyz, bx.size() * 4));
    DG_CUDA(cudaMemcpy(c->bxyz, bx.data(), bx.size() * 4, cudaMemcpyHostToDevice));
    std::vector<int32_t> bf(bfaces.begin(), bfaces.end());
    DG_CUDA(cudaMalloc(&c->bface, bf.size() * 4));
    DG_CUDA(cudaMemcpy(c->bface, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice));
    c->nbf = int64_t(bfaces.size());
    const size_t nb = bfaces.size() * size_t(Nfp) * 4;
    DG_CUDA(cudaMalloc(&c->bpsi, nb));
    DG_CUDA(cudaMalloc(&c->bpsi_res, nb));
    DG_CUDA(cudaMalloc(&c->bD, nb));
    DG_CUDA(cudaMemset(c->bpsi, 0, nb));
    DG_CUDA(cudaMemset(c->bpsi_res, 0, nb));
    DG_CUDA(cudaMemset(c->bD, 0, nb));
  }
  {
    // faces each tile evaluates: a face shared by two elements of the tile
    // once, under the lower element (the stage writes both jumps). Grouped:
    // faces inside the tile, then faces to other tiles, then outer faces;
    // header int32 {total, inside, to other tiles, 0}
    const size_t row = 16 + (4 * size_t(ET) + 15) / 16 * 16;   // rows start on 16-byte boundaries
    std::vector<uint8_t> fl(size_t(c->ntiles) * row, 0);
    std::vector<uint8_t> grp[3];
    for (int t = 0; t < c->ntiles; ++t) {
      const int64_t e0 = int64_t(t) * ET, e1 = std::min<int64_t>(Kown, e0 + ET);
      for (auto& g : grp) g.clear();
      for (int64_t e = e0; e < e1; ++e)
        for (int f = 0; f < 4; ++f) {
          const int64_t e2 = c->mesh.EToE[size_t(e) * 4 + f];
          const bool inside = e2 >= e0 && e2 < e1;
          if (inside && e2 < e) continue;
          grp[e2 < 0 ? 2 : (inside ? 0 : 1)].push_back(uint8_t(((e - e0) << 2) | f));
        }
      int32_t hdr[4] = {int32_t(grp[0].size() + grp[1].size() + grp[2].size()), int32_t(grp[0].size()),
                        int32_t(grp[1].size()), 0};
      std::memcpy(&fl[size_t(t) * row], hdr, 16);
      size_t pos = size_t(t) * row + 16;
      for (auto& g : grp)
        for (uint8_t b : g) fl[pos++] = b;
    }
    DG_CUDA(cudaMalloc(&c->face_list, fl.size()));
    DG_CUDA(cudaMemcpy(c->face_list, fl.data(), fl.size(), cudaMemcpyHostToDevice));
  }
  DG_CUDA(cudaMalloc(&c->conn, conn.size() * 4));
  DG_CUDA(cudaMemcpy(c->conn, conn.data(), conn.size() * 4, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMalloc(&c->ledger_part, size_t(c->grid) * 5 * 8));
  DG_CUDA(cudaMemset(c->ledger_part, 0, size_t(c->grid) * 5 * 8));
  DG_CUDA(cudaMalloc(&c->ticket, sizeof(unsigned long long)));
  DG_CUDA(cudaMemset(c->ticket, 0, sizeof(unsigned long long)));
  DG_CUDA(cudaMalloc(&c->ledger, 10 * 8));
  DG_CUDA(cudaMemset(c->ledger, 0, 10 * 8));
  // operators, transposed so that consecutive nodes are consecutive words
  std::vector<double> ops(size_t(3) * Np * Np + size_t(NF) * Np + NF);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      ops[size_t(j) * Np + i] = c->ref.Dr[size_t(i) * Np + j];
      ops[size_t(Np) * Np + size_t(j) * Np + i] = c->ref.Ds[size_t(i) * Np + j];
      ops[size_t(2) * Np * Np + size_t(j) * Np + i] = c->ref.Dt[size_t(i) * Np + j];
    }
  for (int i = 0; i < Np; ++i)
    for (int m = 0; m < NF; ++m)
      ops[size_t(3) * Np * Np + size_t(m) * Np + i] = c->ref.LIFT[size_t(i) * NF + m];
  for (int m = 0; m < NF; ++m) ops[size_t(3) * Np * Np + size_t(NF) * Np + m] = c->ref.face_w[m];
  DG_CUDA(cudaMalloc(&c->ops, ops.size() * 8));
  DG_CUDA(cudaMemcpy(c->ops, ops.data(), ops.size() * 8, cudaMemcpyHostToDevice));
  if (modal) {
    dg::ModalOps mo;
    std::string merr;
    if (!dg::build_modal_ops(c->ref, mo, merr)) return c->fail(DG_ERR_ARG, merr);
    std::vector<double> blk;
    blk.insert(blk.end(), mo.Iq.begin(), mo.Iq.end());
    blk.insert(blk.end(), mo.Sv.begin(), mo.Sv.end());
    blk.insert(blk.end(), mo.Ifn.begin(), mo.Ifn.end());
    blk.insert(blk.end(), mo.Sf.begin(), mo.Sf.end());
    for (int q = 0; q < mo.Nfq; ++q) blk.push_back(mo.face[3 * q + 2]);
    if (int(blk.size()) != dgk::modal_ops_len(p))
      return c->fail(DG_ERR_ARG, "modal operator block size mismatch");
    DG_CUDA(cudaMalloc(&c->mops, blk.size() * 8));
    DG_CUDA(cudaMemcpy(c->mops, blk.data(), blk.size() * 8, cudaMemcpyHostToDevice));
  }
  if (tcf) {
    // operator matrix [-Dr | -Ds | -Dt | LIFT] as the tensor-core operand image
    std::vector<unsigned char> img(dgk::stage_tc_ops_bytes(p, c->tc_images()));
    dgk::build_tc_ops(p, c->tc_images(), c->ref.Dr.data(), c->ref.Ds.data(), c->ref.Dt.data(),
                      c->ref.LIFT.data(), c->ref.face_w.data(), img.data());
    DG_CUDA(cudaMalloc(&c->ops32, img.size()));
    DG_CUDA(cudaMemcpy(c->ops32, img.data(), img.size(), cudaMemcpyHostToDevice));
  } else if (f32) {
    std::vector<float> o32(ops.begin(), ops.end());
    DG_CUDA(cudaMalloc(&c->ops32, o32.size() * 4));
    DG_CUDA(cudaMemcpy(c->ops32, o32.data(), o32.size() * 4, cudaMemcpyHostToDevice));
  }
  const std::vector<uint8_t> tbl2 = face_node_tables(c->ref);
  DG_CUDA(cudaMalloc(&c->tbl, tbl2.size()));
  DG_CUDA(cudaMemcpy(c->tbl, tbl2.data(), tbl2.size(),
                     cudaMemcpyHostToDevice));
  std::vector<int32_t> fm(c->ref.Fmask.begin(), c->ref.Fmask.end());
  DG_CUDA(cudaMalloc(&c->fmask, fm.size() * 4));
  DG_CUDA(cudaMemcpy(c->fmask, fm.data(), fm.size() * 4, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMalloc(&c->mass_w, size_t(Np) * 8));
  DG_CUDA(cudaMemcpy(c->mass_w, c->mass_w_host.data(), size_t(Np) * 8, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMalloc(&c->totals_part, size_t(kTotalsBlocks + 1) * 5 * 8));
  DG_CUDA(cudaMalloc(&c->status, sizeof(int)));
  DG_CUDA(cudaMemset(c->status, 0, sizeof(int)));
  c->dev_ready = true;
  return DG_OK;
}

dgk::LedgerArgs ledger_args(dg_ctx* c, bool update, double a, double b, double dt) {
  return dgk::LedgerArgs{c->ledger_part, c->ledger, c->ticket, a, b, dt, update ? 1 : 0};
}

dgk::StageArgs stage_args(dg_ctx* c, const double* qin, double* qout, double* res, double a,
                          double b, double dt, bool update) {
  dgk::StageArgs A{};
  A.q_in = qin;
  A.q_out = qout;
  A.res = res;
  A.geo = c->geo;
  A.conn = c->conn;
  A.ops = c->ops;
  A.nbr_tbl = c->tbl;
  A.fmask = c->fmask;
  A.face_list = c->face_list;
  A.led = ledger_args(c, update, a, b, dt);
  A.status = c->status;
  A.K = c->owned();
  A.K_all = c->mesh.K;
  A.ntiles = c->ntiles;
  for (int i = 0; i < 8; ++i) A.bc_mode[i] = c->bc_mode[i];
  A.a = a;
  A.b = b;
  A.dt = dt;
  A.gas = c->gas;
  return A;
}

dgk::BaseGhost base_ghost(const dg_ctx* c) {
  return dgk::BaseGhost{float(c->gas.rho0), float(c->gas.p0), float(c->gas.gamma), float(c->gas.gm1),
                        float(c->gas.c0)};
}

// Closure increments and memories for the stage about to run (float32 forms):
// learned boundary faces get their increments D (and, in a time step, their
// memory update); trace faces get their memory update while traces are
// recorded. dg_eval_rhs (to_scratch) computes D without advancing anything.
// *launched: whether a kernel went into the stream (the stage kernel is then
// launched as its programmatic dependent).
int run_memory(dg_ctx* c, bool to_scratch, double a, double b, double dt, bool* launched) {
  *launched = false;
  bool learned = false;
  for (int i = 0; i < 8; ++i) learned = learned || c->bc_mode[i] == DG_BC_LEARNED;
  if (learned && c->nbf > 0 && c->mesh.verts.empty())
    return c->fail(DG_ERR_ORDER, "the learned closure needs vertex coordinates (dg_upload_mesh)");
  const dgk::BaseGhost bg = base_ghost(c);
  if (learned && c->nbf > 0) {
    if (c->mlp_w && !c->mlp_img_ok) {
      DG_CUDA(dgk::launch_closure_image(c->mlp_w, c->mlp_img, c->stream));
      c->mlp_img_ok = true;
    }
    dgk::ClosureArgs C{};
    C.q = c->q32[c->cur];
    C.Np = c->ref.Np;
    C.Nfp = c->ref.Nfp;
    C.bface = c->bface;
    C.nb = c->nbf;
    C.conn = c->conn;
    C.fmask = c->fmask;
    C.geo = c->geo32;
    C.bxyz = c->bxyz;
    for (int i = 0; i < 8; ++i) C.bc_mode[i] = c->bc_mode[i];
    C.w = c->mlp_w;
    C.wimg = c->mlp_img;
    C.S = mlp_scales(c);
    C.psi = c->bpsi;
    C.psi_res = c->bpsi_res;
    C.D = c->bD;
    C.a = float(a);
    C.b = float(b);
    C.dt = float(dt);
    C.advance = to_scratch ? 0 : 1;
    C.status = c->status;
    C.K_all = c->mesh.K;
    DG_CUDA(dgk::launch_closure(C, bg, c->stream));
    *launched = C.nb * C.Nfp > 0;
  }
  if (c->ntrace > 0 && !to_scratch) {
    DG_CUDA(dgk::launch_trace_memory(c->q32[c->cur], c->ref.Np, c->ref.Nfp, c->tr_elem, c->tr_face,
                                     c->fmask, c->geo32, c->txyz, c->ntrace, bg, mlp_scales(c),
                                     c->tr_psi, c->tr_res, float(a), float(b), float(dt), c->stream));
    *launched = true;
  }
  return DG_OK;
}

// One Runge-Kutta stage from q[cur] to q[1-cur]; with to_scratch the residual
// goes to the scratch buffer (used by dg_eval_rhs with a = b = 0, dt = 1).
// Inflow ghost (section 2.4, Eqs. 5-7) at time t: pressure p0 (1 + A (1 -
// cos(alpha t))) during one period, rho = rho0 (p/p0)^(1/gamma), speed
// (p - p0)/(rho0 c0) into the domain; as {rho, rho u_in, E} and, for the
// float32 forms, as {rho - rho0, rho u_in, E - E0} formed without cancellation.
void inflow_state(const dg_ctx* c, double t, double full[3], float pert[3]) {
  const dgk::Gas& g = c->gas;
  const double kTwoPi = 6.283185307179586;
  const bool on = t >= 0.0 && t < kTwoPi / c->inflow_alpha;
  const double dp = on ? g.p0 * c->inflow_amp * (1.0 - std::cos(c->inflow_alpha * t)) : 0.0;
  const double drho = g.rho0 * std::expm1(std::log1p(dp / g.p0) / g.gamma);
  const double rho = g.rho0 + drho;
  const double un = dp / (g.rho0 * g.c0);
  const double dE = dp / g.gm1 + 0.5 * rho * un * un;
  full[0] = rho;
  full[1] = rho * un;
  full[2] = (g.p0 + dp) / g.gm1 + 0.5 * rho * un * un;
  pert[0] = float(drho);
  pert[1] = float(rho * un);
  pert[2] = float(dE);
}

int run_stage(dg_ctx* c, bool to_scratch, double a, double b, double dt, double ts) {
  double in_full[3];
  float in_pert[3];
  inflow_state(c, ts, in_full, in_pert);
  if (c->f32()) {
    dgk::StageArgsF32 A{};
    A.q_in = c->q32[c->cur];
    A.q_out = c->q32[1 - c->cur];
    A.res = to_scratch ? c->scratch32 : c->res32;
    A.geo = c->geo32;
    A.conn = c->conn;
    A.ops = c->ops32;
    A.nbr_tbl = c->tbl;
    A.fmask = c->fmask;
    A.led = ledger_args(c, !to_scratch, a, b, dt);
    A.status = c->status;
    A.K = c->owned();
    A.K_all = c->mesh.K;
    A.nb = c->nbf;
    A.ntiles = c->ntiles;
    for (int i = 0; i < 8; ++i) A.bc_mode[i] = c->bc_mode[i];
    A.a = float(a);
    A.b = float(b);
    A.dt = float(dt);
    A.gas = c->gas;
    for (int i = 0; i < 3; ++i) A.inflow[i] = in_pert[i];
    A.bD = c->bD;
    A.face_list = c->face_list;
    bool after_kernel = false;
    int rc = run_memory(c, to_scratch, a, b, dt, &after_kernel);
    if (rc) return rc;
    // the stage kernel may start while the closure finishes: before its
    // griddep_wait (after its prologue) it touches nothing the closure
    // writes (D, the memories) and writes nothing the closure reads
    A.pdl = after_kernel ? 1 : 0;
    if (c->tc())
      DG_CUDA(dgk::launch_stage_tc(c->ref.p, c->tc_images(), A, c->grid, c->stream));
    else
      DG_CUDA(dgk::launch_stage_f32(c->ref.p, A, c->grid, c->stream));
  } else {
    dgk::StageArgs A = stage_args(c, c->q[c->cur], c->q[1 - c->cur], to_scratch ? c->scratch : c->res,
                                  a, b, dt, !to_scratch);
    for (int i = 0; i < 3; ++i) A.inflow[i] = in_full[i];
    if (c->prec == DG_PREC_MODAL) {
      A.modal_ops = c->mops;
      DG_CUDA(dgk::launch_stage_modal(c->ref.p, A, c->grid, c->stream));
    } else {
      DG_CUDA(dgk::launch_stage(c->ref.p, A, c->grid, c->stream));
    }
  }
  return DG_OK;
}

// Total state (float64) of the current solution into the scratch buffer.
int current_state_f64(dg_ctx* c, double* dst) {
  if (c->f32())
    DG_CUDA(dgk::launch_from_perturbation(c->q32[c->cur], dst, c->mesh.K, c->ref.Np, c->gas.rho0,
                                          c->gas.E0, c->stream));
  else if (dst != c->q[c->cur])
    DG_CUDA(cudaMemcpyAsync(dst, c->q[c->cur], c->state_elems() * 8, cudaMemcpyDeviceToDevice,
                            c->stream));
  return DG_OK;
}

// One thread fails a bounds check on purpose (a condition nothing meets):
// the status word's path to the host, tested without an out-of-range access.
__global__ void bounds_selftest_kernel(int* status, unsigned limit) {
  if (!DG_IN(threadIdx.x > limit, status)) return;
}

cudaError_t bounds_selftest(int* status, cudaStream_t s) {
  bounds_selftest_kernel<<<1, 1, 0, s>>>(status, 1024u);
  return cudaGetLastError();
}

int check_status(dg_ctx* c) {
  int st = 0;
  DG_CUDA(cudaStreamSynchronize(c->stream));
  DG_CUDA(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    DG_CUDA(cudaMemset(c->status, 0, sizeof(int)));
    if (st & dgk::kStatusBounds)
      return c->fail(DG_ERR_BOUNDS, "a device bounds check failed (an index read from the mesh "
                                    "tables was out of range; debug build)");
    if (st & dgk::kStatusTimeout)
      return c->fail(DG_ERR_TIMEOUT, "a bounded wait for tensor-core completion gave up");
    return c->fail(DG_ERR_NONFINITE, "device saw a non-finite or non-physical state "
                                     "(density or pressure <= 0)");
  }
  return DG_OK;
}

// Event pair around a stage launch when timing is on.
int record_event(dg_ctx* c) {
  if (!c->timing) return DG_OK;
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    DG_CUDA(cudaEventCreate(&e));
    c->ev_pool.push_back(e);
  }
  DG_CUDA(cudaEventRecord(c->ev_pool[c->ev_used++], c->stream));
  return DG_OK;
}

int reset_run(dg_ctx* c, double t) {
  c->t = t;
  c->stage_k = 0;
  c->have_state = true;
  c->precorded = 0;
  DG_CUDA(cudaMemsetAsync(c->ledger, 0, 10 * 8, c->stream));
  // a new run starts with empty memories
  const size_t nb = size_t(c->nbf) * c->ref.Nfp * 4, nt = size_t(c->ntrace) * c->ref.Nfp * 4;
  if (nb) {
    DG_CUDA(cudaMemsetAsync(c->bpsi, 0, nb, c->stream));
    DG_CUDA(cudaMemsetAsync(c->bpsi_res, 0, nb, c->stream));
  }
  if (nt) {
    DG_CUDA(cudaMemsetAsync(c->tr_psi, 0, nt, c->stream));
    DG_CUDA(cudaMemsetAsync(c->tr_res, 0, nt, c->stream));
  }
  return DG_OK;
}

}  // namespace

extern "C" {

int dg_create(int order, const dg_params* params, dg_ctx** out) {
  if (!out) return DG_ERR_ARG;
  *out = nullptr;
  if (!params) return DG_ERR_ARG;
  if (!(params->gamma > 1.0) || !(params->rho0 > 0.0) || !(params->p0 > 0.0)) return DG_ERR_ARG;
  if (params->default_bc < 0 || params->default_bc > 2) return DG_ERR_ARG;
  if (params->precision != DG_PREC_FP64 && params->precision != DG_PREC_F32 &&
      params->precision != DG_PREC_F32_TC && params->precision != DG_PREC_MODAL &&
      params->precision != DG_PREC_F32_TC1)
    return DG_ERR_UNSUPPORTED;
  if ((params->precision == DG_PREC_F32 || params->precision == DG_PREC_F32_TC ||
       params->precision == DG_PREC_F32_TC1) &&
      (params->u0[0] != 0.0 || params->u0[1] != 0.0 || params->u0[2] != 0.0))
    return DG_ERR_UNSUPPORTED;   // the perturbation form is built around a resting base state
  if (order < 1 || order > dg::kMaxOrder) return DG_ERR_UNSUPPORTED;
  dg_ctx* c = new (std::nothrow) dg_ctx();
  if (!c) return DG_ERR_ARG;
  std::string err;
  if (!dg::build_ref_element(order, c->ref, err)) {
    delete c;
    return DG_ERR_ARG;
  }
  c->prm = *params;
  c->prec = params->precision;
  for (int i = 0; i < 8; ++i) c->bc_mode[i] = params->default_bc;
  dgk::Gas& g = c->gas;
  g.gamma = params->gamma;
  g.gm1 = params->gamma - 1.0;
  g.rho0 = params->rho0;
  g.p0 = params->p0;
  for (int d = 0; d < 3; ++d) g.u0[d] = params->u0[d];
  g.c0 = std::sqrt(g.gamma * g.p0 / g.rho0);
  g.E0 = g.p0 / g.gm1 + 0.5 * g.rho0 * (g.u0[0] * g.u0[0] + g.u0[1] * g.u0[1] + g.u0[2] * g.u0[2]);
  g.s_inf = g.p0 / std::pow(g.rho0, g.gamma);
  // mass-matrix column sums 1^T M with M = (V V^T)^-1 = invV^T invV
  const int Np = c->ref.Np;
  c->mass_w_host.assign(Np, 0.0);
  for (int j = 0; j < Np; ++j) {
    double s = 0.0;
    for (int i = 0; i < Np; ++i)
      for (int m = 0; m < Np; ++m) s += c->ref.invV[size_t(m) * Np + i] * c->ref.invV[size_t(m) * Np + j];
    c->mass_w_host[j] = s;
  }
  *out = c;
  return DG_OK;
}

int dg_destroy(dg_ctx* c) {
  if (!c) return DG_OK;
  c->free_device();
  dfree(c->mlp_img); dfree(c->mlp_w); dfree(c->mlp_m); dfree(c->mlp_v); dfree(c->mlp_grad); dfree(c->mlp_loss);
  dfree(c->mlp_part);
  delete c;
  return DG_OK;
}

const char* dg_last_error(const dg_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

int dg_set_stream(dg_ctx* c, void* stream) {
  if (!c) return DG_ERR_ARG;
  if (c->dev_ready) cudaStreamSynchronize(c->stream);
  c->stream = static_cast<cudaStream_t>(stream);
  return DG_OK;
}

int dg_upload_mesh(dg_ctx* c, int64_t nvert, const double* xyz, int64_t K, const int32_t* EToV,
                   const int8_t* face_tag, const int64_t* vert_class) {
  if (!c) return DG_ERR_ARG;
  if (K <= 0 || nvert <= 0 || !xyz || !EToV) return c->fail(DG_ERR_ARG, "empty mesh or null array");
  if (K > (int64_t(1) << 26)) return c->fail(DG_ERR_ARG, "too many elements (max 2^26)");
  c->free_device();
  c->have_mesh = false;
  c->K_own = -1;
  std::string err;
  if (!dg::build_mesh(c->ref, nvert, xyz, K, EToV, face_tag, vert_class, c->mesh, err))
    return c->fail(DG_ERR_MESH, err);
  c->have_mesh = true;
  return DG_OK;
}

int dg_upload_geometry(dg_ctx* c, int64_t K, const double* drdx, const double* J,
                       const double* nrm, const double* Fscale, const int32_t* EToE,
                       const int8_t* EToF, const int8_t* orient, const int8_t* bc) {
  if (!c) return DG_ERR_ARG;
  if (K <= 0 || !drdx || !J || !nrm || !Fscale || !EToE || !EToF || !orient)
    return c->fail(DG_ERR_ARG, "empty mesh or null array");
  if (K > (int64_t(1) << 26)) return c->fail(DG_ERR_ARG, "too many elements (max 2^26)");
  c->free_device();
  c->have_mesh = false;
  c->K_own = -1;
  dg::Mesh m;
  m.K = K;
  m.drdx.assign(drdx, drdx + size_t(K) * 9);
  m.J.assign(J, J + K);
  m.nrm.assign(nrm, nrm + size_t(K) * 12);
  m.Fscale.assign(Fscale, Fscale + size_t(K) * 4);
  m.EToE.assign(EToE, EToE + size_t(K) * 4);
  m.EToF.assign(size_t(K) * 4, 0);
  m.orient.assign(size_t(K) * 4, 0);
  m.bc.assign(size_t(K) * 4, -1);
  m.sJ.resize(size_t(K) * 4);
  m.rin.resize(K);
  for (int64_t e = 0; e < K; ++e) {
    if (!(J[e] > 0.0) || !std::isfinite(J[e]))
      return c->fail(DG_ERR_MESH, "J <= 0 at element " + std::to_string(e));
    double fsum = 0.0;
    for (int f = 0; f < 4; ++f) {
      const size_t i = size_t(e) * 4 + f;
      const double* n = nrm + i * 3;
      const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      if (!(std::fabs(len - 1.0) < 1e-6))
        return c->fail(DG_ERR_MESH, "normal not of unit length at element " + std::to_string(e));
      if (!(Fscale[i] > 0.0) || !std::isfinite(Fscale[i]))
        return c->fail(DG_ERR_MESH, "Fscale <= 0 at element " + std::to_string(e));
      m.sJ[i] = Fscale[i] * J[e];
      fsum += Fscale[i];
      const int32_t e2 = EToE[i];
      if (e2 < 0) {
        const int8_t tag = bc ? bc[i] : int8_t(0);
        if (tag < 0 || tag > 7) return c->fail(DG_ERR_MESH, "boundary id out of 0..7");
        m.bc[i] = tag;
        continue;
      }
      const int f2 = EToF[i], o = orient[i];
      if (e2 >= K || f2 < 0 || f2 > 3 || o < 0 || o > 5)
        return c->fail(DG_ERR_MESH, "neighbour, face or orientation out of range at element " +
                                        std::to_string(e));
      const size_t j = size_t(e2) * 4 + f2;
      if (EToE[j] != e || EToF[j] != f || orient[j] < 0 || orient[j] > 5)
        return c->fail(DG_ERR_MESH, "neighbour links not mutual at element " + std::to_string(e));
      for (int q = 0; q < 3; ++q)
        if (dg::kPerm[orient[j]][dg::kPerm[o][q]] != q)
          return c->fail(DG_ERR_MESH, "orientation codes not inverse at element " + std::to_string(e));
      const double* n2 = nrm + j * 3;
      if (n[0] * n2[0] + n[1] * n2[1] + n[2] * n2[2] > -1.0 + 1e-6)
        return c->fail(DG_ERR_MESH, "matched faces not back to back at element " + std::to_string(e));
      m.EToF[i] = int8_t(f2);
      m.orient[i] = int8_t(o);
    }
    m.rin[e] = 2.0 / fsum;            // 3 V / total area with V = 4 J / 3, area_f = 2 Fscale_f J
  }
  c->mesh = std::move(m);
  c->have_mesh = true;
  return DG_OK;
}

int dg_set_inflow(dg_ctx* c, double amplitude, double alpha) {
  if (!c) return DG_ERR_ARG;
  if (!std::isfinite(amplitude) || !(alpha > 0.0) || !std::isfinite(alpha) || amplitude <= -0.5)
    return c->fail(DG_ERR_ARG, "need alpha > 0 and amplitude > -1/2");
  c->inflow_amp = amplitude;
  c->inflow_alpha = alpha;
  return DG_OK;
}

int dg_set_bc(dg_ctx* c, int bc_id, int mode) {
  if (!c) return DG_ERR_ARG;
  if (bc_id < 0 || bc_id > 7) return c->fail(DG_ERR_ARG, "boundary id must be 0..7");
  if (mode < 0 || mode > 4) return c->fail(DG_ERR_ARG, "unknown boundary mode");
  if (mode == DG_BC_LEARNED && !c->f32())
    return c->fail(DG_ERR_UNSUPPORTED, "the learned closure runs in the float32 forms");
  c->bc_mode[bc_id] = mode;
  return DG_OK;
}

int dg_sizes(const dg_ctx* c, int64_t* K, int32_t* Np, int32_t* Nfp) {
  if (!c) return DG_ERR_ARG;
  if (K) *K = c->have_mesh ? c->mesh.K : 0;
  if (Np) *Np = c->ref.Np;
  if (Nfp) *Nfp = c->ref.Nfp;
  return DG_OK;
}

int dg_node_coords(const dg_ctx* c, double* xyz) {
  if (!c || !xyz) return DG_ERR_ARG;
  if (!c->have_mesh || c->mesh.verts.empty()) return DG_ERR_ORDER;
  const int Np = c->ref.Np;
  for (int64_t e = 0; e < c->mesh.K; ++e) {
    const double* v = &c->mesh.verts[size_t(e) * 12];
    for (int n = 0; n < Np; ++n) {
      const double r = c->ref.r[n], s = c->ref.s[n], t = c->ref.t[n];
      const double w[4] = {-0.5 * (1 + r + s + t), 0.5 * (1 + r), 0.5 * (1 + s), 0.5 * (1 + t)};
      for (int d = 0; d < 3; ++d)
        xyz[(size_t(e) * Np + n) * 3 + d] =
            w[0] * v[d] + w[1] * v[3 + d] + w[2] * v[6 + d] + w[3] * v[9 + d];
    }
  }
  return DG_OK;
}

int dg_get_geometry(const dg_ctx* c, double* J, double* drdx, double* nrm, double* sJ,
                    int32_t* EToE, int8_t* EToF, int8_t* bc) {
  if (!c) return DG_ERR_ARG;
  if (!c->have_mesh) return DG_ERR_ORDER;
  const dg::Mesh& m = c->mesh;
  if (J) std::memcpy(J, m.J.data(), m.J.size() * 8);
  if (drdx) std::memcpy(drdx, m.drdx.data(), m.drdx.size() * 8);
  if (nrm) std::memcpy(nrm, m.nrm.data(), m.nrm.size() * 8);
  if (sJ) std::memcpy(sJ, m.sJ.data(), m.sJ.size() * 8);
  if (EToE) std::memcpy(EToE, m.EToE.data(), m.EToE.size() * 4);
  if (EToF) std::memcpy(EToF, m.EToF.data(), m.EToF.size());
  if (bc) std::memcpy(bc, m.bc.data(), m.bc.size());
  return DG_OK;
}

int dg_face_pairs(const dg_ctx* c, int64_t* vol_node, int32_t* face_node) {
  if (!c) return DG_ERR_ARG;
  if (!c->have_mesh) return DG_ERR_ORDER;
  const int Np = c->ref.Np, Nfp = c->ref.Nfp;
  const std::vector<uint8_t> tbl = face_node_tables(c->ref);
  const size_t half = tbl.size() / 2;
  for (int64_t e = 0; e < c->mesh.K; ++e)
    for (int f = 0; f < 4; ++f) {
      const size_t i = size_t(e) * 4 + f;
      const bool inner = c->mesh.EToE[i] >= 0;
      // decoded from the connection word exactly as the stage kernels do
      const int32_t w = inner ? dgk::conn_interior(c->mesh.EToE[i], c->mesh.EToF[i], c->mesh.orient[i]) : 0;
      const int64_t e2 = w >> 5;
      const int f2 = (w >> 3) & 3, o = w & 7;
      for (int m = 0; m < Nfp; ++m) {
        const size_t t = ((size_t(f) * 4 + f2) * 6 + o) * Nfp + m, out = i * Nfp + m;
        if (vol_node) vol_node[out] = inner ? e2 * Np + tbl[t] : -1;
        if (face_node) face_node[out] = inner ? int32_t(tbl[half + t]) : -1;
      }
    }
  return DG_OK;
}

int dg_stable_dt(const dg_ctx* c, const double* q, double cfl, double* dt) {
  if (!c || !q || !dt || !(cfl > 0.0)) return DG_ERR_ARG;
  if (!c->have_mesh) return DG_ERR_ORDER;
  const int Np = c->ref.Np;
  const double g = c->prm.gamma;
  double smax = 0.0, rmin = 1e300;
  for (int64_t e = 0; e < c->mesh.K; ++e) {
    rmin = std::min(rmin, c->mesh.rin[e]);
    for (int n = 0; n < Np; ++n) {
      const double* b = q + size_t(e) * 5 * Np + n;
      const double rho = b[0], mx = b[Np], my = b[2 * Np], mz = b[3 * Np], E = b[4 * Np];
      const double u2 = (mx * mx + my * my + mz * mz) / (rho * rho);
      const double p = (g - 1.0) * (E - 0.5 * rho * u2);
      if (!(rho > 0.0) || !(p > 0.0)) return DG_ERR_ARG;
      smax = std::max(smax, std::sqrt(u2) + std::sqrt(g * p / rho));
    }
  }
  const int p1 = c->ref.p + 1;
  *dt = cfl * rmin / (double(p1) * p1 * smax);
  return DG_OK;
}

int dg_reference_operators(int order, double* rst, double* Dr, double* Ds, double* Dt,
                           double* LIFT, int32_t* Fmask) {
  dg::RefElement re;
  std::string err;
  if (!dg::build_ref_element(order, re, err)) return DG_ERR_UNSUPPORTED;
  const int Np = re.Np;
  if (rst) {
    std::memcpy(rst, re.r.data(), Np * 8);
    std::memcpy(rst + Np, re.s.data(), Np * 8);
    std::memcpy(rst + 2 * Np, re.t.data(), Np * 8);
  }
  if (Dr) std::memcpy(Dr, re.Dr.data(), re.Dr.size() * 8);
  if (Ds) std::memcpy(Ds, re.Ds.data(), re.Ds.size() * 8);
  if (Dt) std::memcpy(Dt, re.Dt.data(), re.Dt.size() * 8);
  if (LIFT) std::memcpy(LIFT, re.LIFT.data(), re.LIFT.size() * 8);
  if (Fmask)
    for (size_t i = 0; i < re.Fmask.size(); ++i) Fmask[i] = re.Fmask[i];
  return DG_OK;
}

int dg_modal_quadrature(int order, double* vol, double* face, int32_t* nq, int32_t* nfq) {
  if (order < 1 || order > dg::kMaxOrder) return DG_ERR_UNSUPPORTED;
  std::vector<double> v, f;
  dg::tet_rule(2 * order, v);
  dg::tri_rule(2 * order + 1, f);
  if (vol) std::memcpy(vol, v.data(), v.size() * 8);
  if (face) std::memcpy(face, f.data(), f.size() * 8);
  if (nq) *nq = int32_t(v.size() / 4);
  if (nfq) *nfq = int32_t(f.size() / 3);
  return DG_OK;
}

int dg_modal_operators(int order, double* Iq, double* Sv, double* Ifn, double* Sf, double* wf) {
  dg::RefElement re;
  std::string err;
  if (!dg::build_ref_element(order, re, err)) return DG_ERR_UNSUPPORTED;
  dg::ModalOps mo;
  if (!dg::build_modal_ops(re, mo, err)) return DG_ERR_ARG;
  if (Iq) std::memcpy(Iq, mo.Iq.data(), mo.Iq.size() * 8);
  if (Sv) std::memcpy(Sv, mo.Sv.data(), mo.Sv.size() * 8);
  if (Ifn) std::memcpy(Ifn, mo.Ifn.data(), mo.Ifn.size() * 8);
  if (Sf) std::memcpy(Sf, mo.Sf.data(), mo.Sf.size() * 8);
  if (wf)
    for (int q = 0; q < mo.Nfq; ++q) wf[q] = mo.face[3 * q + 2];
  return DG_OK;
}

int dg_set_state(dg_ctx* c, const double* q, double t) {
  if (!c || !q) return DG_ERR_ARG;
  int rc = ensure_device(c);
  if (rc) return rc;
  if (c->f32()) {
    DG_CUDA(cudaMemcpyAsync(c->scratch, q, c->state_elems() * 8, cudaMemcpyHostToDevice, c->stream));
    DG_CUDA(dgk::launch_to_perturbation(c->scratch, c->q32[c->cur], c->mesh.K, c->ref.Np,
                                        c->gas.rho0, c->gas.E0, c->stream));
  } else {
    DG_CUDA(cudaMemcpyAsync(c->q[c->cur], q, c->state_elems() * 8, cudaMemcpyHostToDevice, c->stream));
  }
  return reset_run(c, t);
}

int dg_set_state_device(dg_ctx* c, const double* dq, double t) {
  if (!c || !dq) return DG_ERR_ARG;
  int rc = ensure_device(c);
  if (rc) return rc;
  if (c->f32())
    DG_CUDA(dgk::launch_to_perturbation(dq, c->q32[c->cur], c->mesh.K, c->ref.Np, c->gas.rho0,
                                        c->gas.E0, c->stream));
  else
    DG_CUDA(cudaMemcpyAsync(c->q[c->cur], dq, c->state_elems() * 8, cudaMemcpyDeviceToDevice, c->stream));
  return reset_run(c, t);
}

int dg_get_state(dg_ctx* c, double* q, double* t) {
  if (!c || !q) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  const double* src = c->q[c->cur];
  if (c->f32()) {
    int rc = current_state_f64(c, c->scratch);
    if (rc) return rc;
    src = c->scratch;
  }
  DG_CUDA(cudaMemcpyAsync(q, src, c->state_elems() * 8, cudaMemcpyDeviceToHost, c->stream));
  if (t) *t = c->t;
  return check_status(c);
}

int dg_get_state_device(dg_ctx* c, double* dq, double* t) {
  if (!c || !dq) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  int rc = current_state_f64(c, dq);
  if (rc) return rc;
  if (t) *t = c->t;
  return DG_OK;
}

// Advance n Runge-Kutta stages from the stage counter on; after the last
// stage of a step the time advances and the sensors are sampled.
static int advance_stages(dg_ctx* c, int64_t n, double dt) {
  const bool heun = c->prec == DG_PREC_MODAL;
  const int nstage = heun ? 2 : 5;
  const double* RA = heun ? kHeunA : kRkA;
  const double* RB = heun ? kHeunB : kRkB;
  const double* RC = heun ? kHeunC : kRkC;
  for (int64_t s = 0; s < n; ++s) {
    const int k = c->stage_k;
    int rc = record_event(c);
    if (rc) return rc;
    rc = run_stage(c, false, RA[k], RB[k], dt, c->t + RC[k] * dt);
    if (rc) return rc;
    rc = record_event(c);
    if (rc) return rc;
    c->cur = 1 - c->cur;
    c->stage_k = (k + 1) % nstage;
    if (c->stage_k != 0) continue;
    c->t += dt;
    if (c->nprobe > 0) {
      const int slotp = int(c->precorded % c->pcap);
      double* dst = c->pring + size_t(slotp) * c->nprobe * 5;
      if (c->f32())
        DG_CUDA(dgk::launch_probe_sample_f32(c->q32[c->cur], c->ref.Np, c->nprobe, c->pelem, c->prow,
                                             c->gas.rho0, c->gas.E0, dst, c->stream));
      else
        DG_CUDA(dgk::launch_probe_sample(c->q[c->cur], c->ref.Np, c->nprobe, c->pelem, c->prow, dst,
                                         c->stream));
      ++c->precorded;
    }
  }
  return DG_OK;
}

int dg_step(dg_ctx* c, int n, double dt) {
  if (!c) return DG_ERR_ARG;
  if (n < 0 || !(dt > 0.0) || !std::isfinite(dt)) return c->fail(DG_ERR_ARG, "need n >= 0 and dt > 0");
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  if (c->stage_k != 0) return c->fail(DG_ERR_ORDER, "a step is in progress (dg_step_stages)");
  // a named range per call for timeline tools (no cost without one attached)
  struct Range {
    Range() { nvtxRangePushA("dg_step"); }
    ~Range() { nvtxRangePop(); }
  } range;
  return advance_stages(c, int64_t(n) * (c->prec == DG_PREC_MODAL ? 2 : 5), dt);
}

int dg_step_stages(dg_ctx* c, int n, double dt) {
  if (!c) return DG_ERR_ARG;
  if (n < 0 || !(dt > 0.0) || !std::isfinite(dt)) return c->fail(DG_ERR_ARG, "need n >= 0 and dt > 0");
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  return advance_stages(c, n, dt);
}

int dg_stage_index(dg_ctx* c, int* k, int* stages_per_step) {
  if (!c || !k || !stages_per_step) return DG_ERR_ARG;
  *k = c->stage_k;
  *stages_per_step = c->prec == DG_PREC_MODAL ? 2 : 5;
  return DG_OK;
}

int dg_set_owned(dg_ctx* c, int64_t K_own) {
  if (!c) return DG_ERR_ARG;
  if (!c->have_mesh) return c->fail(DG_ERR_ORDER, "no mesh uploaded");
  if (K_own < 1 || K_own > c->mesh.K) return c->fail(DG_ERR_ARG, "need 1 <= K_own <= K");
  if (c->prec == DG_PREC_MODAL)
    return c->fail(DG_ERR_UNSUPPORTED,
                   "the paper's discretisation ties its face rule to the element numbering; "
                   "partitioned meshes run the nodal forms");
  c->free_device();
  c->K_own = K_own;
  return DG_OK;
}

int dg_set_halo(dg_ctx* c, int64_t n_send, const int32_t* send_elem, const int8_t* send_face,
                int64_t n_recv, const int32_t* recv_elem, const int8_t* recv_face) {
  if (!c) return DG_ERR_ARG;
  if (!c->have_mesh) return c->fail(DG_ERR_ORDER, "no mesh uploaded");
  if (n_send < 0 || n_recv < 0 || (n_send > 0 && (!send_elem || !send_face)) ||
      (n_recv > 0 && (!recv_elem || !recv_face)))
    return c->fail(DG_ERR_ARG, "bad halo list arguments");
  const int64_t Kown = c->owned();
  std::vector<int32_t> snd(static_cast<size_t>(n_send)), rcv(static_cast<size_t>(n_recv));
  for (int64_t i = 0; i < n_send; ++i) {
    const int32_t e = send_elem[i];
    const int f = send_face[i];
    if (e < 0 || e >= Kown || f < 0 || f > 3)
      return c->fail(DG_ERR_ARG, "send entry " + std::to_string(i) + " is not a face of an own element");
    if (c->mesh.EToE[size_t(e) * 4 + f] < Kown)
      return c->fail(DG_ERR_ARG, "send entry " + std::to_string(i) + " is not a face to a halo element");
    snd[size_t(i)] = e * 4 + f;
  }
  for (int64_t i = 0; i < n_recv; ++i) {
    const int32_t e = recv_elem[i];
    const int f = recv_face[i];
    if (e < Kown || e >= c->mesh.K || f < 0 || f > 3)
      return c->fail(DG_ERR_ARG, "receive entry " + std::to_string(i) + " is not a face of a halo element");
    const int64_t nb = c->mesh.EToE[size_t(e) * 4 + f];
    if (nb < 0 || nb >= Kown)
      return c->fail(DG_ERR_ARG, "receive entry " + std::to_string(i) + " is not a face to an own element");
    rcv[size_t(i)] = e * 4 + f;
  }
  dfree(c->halo_send);
  dfree(c->halo_recv);
  c->n_send = c->n_recv = 0;
  if (n_send > 0) {
    DG_CUDA(cudaMalloc(&c->halo_send, snd.size() * 4));
    DG_CUDA(cudaMemcpy(c->halo_send, snd.data(), snd.size() * 4, cudaMemcpyHostToDevice));
  }
  if (n_recv > 0) {
    DG_CUDA(cudaMalloc(&c->halo_recv, rcv.size() * 4));
    DG_CUDA(cudaMemcpy(c->halo_recv, rcv.data(), rcv.size() * 4, cudaMemcpyHostToDevice));
  }
  c->n_send = n_send;
  c->n_recv = n_recv;
  return DG_OK;
}

int dg_halo_pack(dg_ctx* c, void* buf) {
  if (!c) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  if (c->n_send == 0) return DG_OK;
  if (!buf) return DG_ERR_ARG;
  if (c->f32())
    DG_CUDA(dgk::launch_halo_pack<float>(c->q32[c->cur], c->ref.Np, c->ref.Nfp, c->halo_send,
                                         c->fmask, c->n_send, static_cast<float*>(buf), c->mesh.K,
                                         c->status, c->stream));
  else
    DG_CUDA(dgk::launch_halo_pack<double>(c->q[c->cur], c->ref.Np, c->ref.Nfp, c->halo_send,
                                          c->fmask, c->n_send, static_cast<double*>(buf), c->mesh.K,
                                          c->status, c->stream));
  return DG_OK;
}

int dg_halo_unpack(dg_ctx* c, const void* buf) {
  if (!c) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  if (c->n_recv == 0) return DG_OK;
  if (!buf) return DG_ERR_ARG;
  if (c->f32())
    DG_CUDA(dgk::launch_halo_unpack<float>(c->q32[c->cur], c->ref.Np, c->ref.Nfp, c->halo_recv,
                                           c->fmask, c->n_recv, static_cast<const float*>(buf),
                                           c->mesh.K, c->status, c->stream));
  else
    DG_CUDA(dgk::launch_halo_unpack<double>(c->q[c->cur], c->ref.Np, c->ref.Nfp, c->halo_recv,
                                            c->fmask, c->n_recv, static_cast<const double*>(buf),
                                            c->mesh.K, c->status, c->stream));
  return DG_OK;
}

int dg_eval_rhs(dg_ctx* c, double* rhs) {
  if (!c || !rhs) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  // one stage with a = b = 0, dt = 1 writes f(q) into the scratch residual
  // and leaves the ledger alone
  int rc = run_stage(c, true, 0.0, 0.0, 1.0, c->t);
  if (rc) return rc;
  if (c->f32())
    DG_CUDA(dgk::launch_widen(c->scratch32, c->scratch, int64_t(c->state_elems()), c->stream));
  DG_CUDA(cudaMemcpyAsync(rhs, c->scratch, c->state_elems() * 8, cudaMemcpyDeviceToHost, c->stream));
  return check_status(c);
}

int dg_set_probes(dg_ctx* c, int n, const double* xyz, int capacity) {
  if (!c) return DG_ERR_ARG;
  if (n < 0 || n > 4096 || (n > 0 && (!xyz || capacity < 1))) return c->fail(DG_ERR_ARG, "bad probe arguments");
  if (n > 0 && (!c->have_mesh || c->mesh.verts.empty()))
    return c->fail(DG_ERR_ORDER, "probes need a mesh with vertex coordinates");
  int rc = ensure_device(c);
  if (rc) return rc;
  DG_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c->pelem); dfree(c->prow); dfree(c->pring);
  c->nprobe = 0;
  c->precorded = 0;
  if (n == 0) return DG_OK;
  const int Np = c->ref.Np;
  std::vector<int32_t> elem(n);
  std::vector<double> rows(size_t(n) * Np);
  for (int i = 0; i < n; ++i) {
    const double* x = xyz + 3 * i;
    int64_t found = -1;
    double rst[3] = {0, 0, 0};
    for (int64_t e = 0; e < c->owned() && found < 0; ++e) {
      const double* v = &c->mesh.verts[size_t(e) * 12];
      const double* m = &c->mesh.drdx[size_t(e) * 9];
      // (r,s,t) = -1 + drdx (x - v1) * ... : r_a + 1 = sum_b drdx[a][b] (x_b - v1_b)
      double ref[3];
      for (int a = 0; a < 3; ++a)
        ref[a] = -1.0 + m[a * 3] * (x[0] - v[0]) + m[a * 3 + 1] * (x[1] - v[1]) + m[a * 3 + 2] * (x[2] - v[2]);
      const double l2 = 0.5 * (1 + ref[0]), l3 = 0.5 * (1 + ref[1]), l4 = 0.5 * (1 + ref[2]);
      const double l1 = 1.0 - l2 - l3 - l4;
      const double tol = -1e-12;
      if (l1 >= tol && l2 >= tol && l3 >= tol && l4 >= tol) {
        found = e;
        rst[0] = ref[0]; rst[1] = ref[1]; rst[2] = ref[2];
      }
    }
    if (found < 0) return c->fail(DG_ERR_ARG, "probe " + std::to_string(i) + " lies outside the mesh");
    elem[i] = int32_t(found);
    // Lagrange basis at the point: l_j(x) = sum_m psi_m(x) invV[m][j]
    std::vector<double> psi(Np);
    dg::eval_basis(c->ref.p, 1, &rst[0], &rst[1], &rst[2], psi.data());
    for (int j = 0; j < Np; ++j) {
      double s = 0.0;
      for (int m2 = 0; m2 < Np; ++m2) s += psi[m2] * c->ref.invV[size_t(m2) * Np + j];
      rows[size_t(i) * Np + j] = s;
    }
  }
  DG_CUDA(cudaMalloc(&c->pelem, size_t(n) * 4));
  DG_CUDA(cudaMalloc(&c->prow, rows.size() * 8));
  DG_CUDA(cudaMalloc(&c->pring, size_t(capacity) * n * 5 * 8));
  DG_CUDA(cudaMemcpy(c->pelem, elem.data(), size_t(n) * 4, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(c->prow, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice));
  c->nprobe = n;
  c->pcap = capacity;
  return DG_OK;
}

int dg_read_probes(dg_ctx* c, int max_steps, double* out, int* got) {
  if (!c || !got || max_steps < 0 || (max_steps > 0 && !out)) return DG_ERR_ARG;
  *got = 0;
  if (c->nprobe == 0) return DG_OK;
  int rc = check_status(c);
  if (rc) return rc;
  const int64_t avail = std::min<int64_t>(c->precorded, c->pcap);
  const int take = int(std::min<int64_t>(avail, max_steps));
  const size_t row = size_t(c->nprobe) * 5;
  for (int i = 0; i < take; ++i) {
    const int64_t step = c->precorded - take + i;
    const int slotp = int(step % c->pcap);
    DG_CUDA(cudaMemcpy(out + size_t(i) * row, c->pring + size_t(slotp) * row, row * 8,
                       cudaMemcpyDeviceToHost));
  }
  c->precorded = 0;
  *got = take;
  return DG_OK;
}

int dg_read_boundary_flux(dg_ctx* c, double out[5]) {
  if (!c || !out) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  int rc = check_status(c);
  if (rc) return rc;
  DG_CUDA(cudaMemcpy(out, c->ledger, 5 * 8, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int dg_conserved_totals(dg_ctx* c, double out[5]) {
  if (!c || !out) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  const double* src = c->q[c->cur];
  if (c->f32()) {
    int rc = current_state_f64(c, c->scratch);
    if (rc) return rc;
    src = c->scratch;
  }
  DG_CUDA(dgk::launch_totals(src, c->geo, c->mass_w, c->owned(), c->ref.Np, c->totals_part,
                             kTotalsBlocks, c->totals_part + size_t(kTotalsBlocks) * 5, c->stream));
  int rc = check_status(c);
  if (rc) return rc;
  DG_CUDA(cudaMemcpy(out, c->totals_part + size_t(kTotalsBlocks) * 5, 5 * 8, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int dg_build_flags(int* flags) {
  if (!flags) return DG_ERR_ARG;
  *flags = dgk::kBoundsChecked ? DG_BUILD_BOUNDS_CHECKS : 0;
  return DG_OK;
}

int dg_bounds_selftest(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  if (!dgk::kBoundsChecked) return c->fail(DG_ERR_UNSUPPORTED, "release build: no bounds checks");
  int rc = ensure_device(c);
  if (rc) return rc;
  DG_CUDA(bounds_selftest(c->status, c->stream));
  return DG_OK;
}

int dg_sync(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  if (!c->dev_ready) return DG_OK;
  return check_status(c);
}

int dg_set_kernel_timing(dg_ctx* c, int enable) {
  if (!c) return DG_ERR_ARG;
  if (c->dev_ready) cudaStreamSynchronize(c->stream);
  c->ev_used = 0;
  c->timing = enable != 0;
  return DG_OK;
}

int dg_read_kernel_timing(dg_ctx* c, double* total_ms, int64_t* launches) {
  if (!c || !total_ms || !launches) return DG_ERR_ARG;
  *total_ms = 0.0;
  *launches = 0;
  if (c->ev_used == 0) return DG_OK;
  DG_CUDA(cudaStreamSynchronize(c->stream));
  double sum = 0.0;
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    DG_CUDA(cudaEventElapsedTime(&ms, c->ev_pool[i], c->ev_pool[i + 1]));
    sum += ms;
  }
  *total_ms = sum;
  *launches = int64_t(c->ev_used / 2);
  c->ev_used = 0;
  return DG_OK;
}

// ------------------------------------------------------- learned closure

int dg_reference_mass(int order, double* M) {
  dg::RefElement re;
  std::string err;
  if (!M) return DG_ERR_ARG;
  if (!dg::build_ref_element(order, re, err)) return DG_ERR_UNSUPPORTED;
  const int Np = re.Np;
  // M = (V V^T)^-1 = invV^T invV for the orthonormal basis
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double s = 0.0;
      for (int m = 0; m < Np; ++m) s += re.invV[size_t(m) * Np + i] * re.invV[size_t(m) * Np + j];
      M[size_t(i) * Np + j] = s;
    }
  return DG_OK;
}

static int ensure_mlp(dg_ctx* c) {
  if (c->mlp_w) return DG_OK;
  const size_t n = dgk::mlp::kParams;
  DG_CUDA(cudaMalloc(&c->mlp_w, n * 4));
  DG_CUDA(cudaMalloc(&c->mlp_m, n * 4));
  DG_CUDA(cudaMalloc(&c->mlp_v, n * 4));
  DG_CUDA(cudaMalloc(&c->mlp_grad, n * 4));
  DG_CUDA(cudaMalloc(&c->mlp_loss, 8));
  DG_CUDA(cudaMalloc(&c->mlp_img, dgk::closure_image_bytes()));
  DG_CUDA(dgk::mlp_prepare());
  DG_CUDA(cudaMemset(c->mlp_w, 0, n * 4));
  DG_CUDA(cudaMemset(c->mlp_img, 0, dgk::closure_image_bytes()));
  c->mlp_img_ok = false;
  return DG_OK;
}

int dg_set_bc_mlp(dg_ctx* c, const float* w, double radius) {
  if (!c || !w || !(radius > 0.0)) return DG_ERR_ARG;
  int rc = ensure_mlp(c);
  if (rc) return rc;
  if (c->dev_ready) DG_CUDA(cudaStreamSynchronize(c->stream));
  DG_CUDA(cudaMemcpy(c->mlp_w, w, size_t(dgk::mlp::kParams) * 4, cudaMemcpyHostToDevice));
  c->mlp_img_ok = false;
  DG_CUDA(cudaMemset(c->mlp_m, 0, size_t(dgk::mlp::kParams) * 4));
  DG_CUDA(cudaMemset(c->mlp_v, 0, size_t(dgk::mlp::kParams) * 4));
  c->mlp_t = 0;
  c->mlp_radius = radius;
  return DG_OK;
}

int dg_get_bc_mlp(dg_ctx* c, float* w) {
  if (!c || !w) return DG_ERR_ARG;
  if (!c->mlp_w) return c->fail(DG_ERR_ORDER, "no network set");
  if (c->dev_ready) DG_CUDA(cudaStreamSynchronize(c->stream));
  DG_CUDA(cudaMemcpy(w, c->mlp_w, size_t(dgk::mlp::kParams) * 4, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int dg_set_trace_faces(dg_ctx* c, int64_t n, const int32_t* elem, const int8_t* face) {
  if (!c || n < 0 || (n > 0 && (!elem || !face))) return DG_ERR_ARG;
  if (!c->f32()) return c->fail(DG_ERR_UNSUPPORTED, "traces are sampled in the float32 forms");
  if (c->have_mesh && c->mesh.verts.empty())
    return c->fail(DG_ERR_ORDER, "trace recording needs vertex coordinates (dg_upload_mesh)");
  int rc = ensure_device(c);
  if (rc) return rc;
  const int Nfp = c->ref.Nfp;
  std::vector<float> xyz(size_t(n) * Nfp * 3);
  for (int64_t t = 0; t < n; ++t) {
    if (elem[t] < 0 || elem[t] >= c->mesh.K || face[t] < 0 || face[t] > 3)
      return c->fail(DG_ERR_ARG, "trace face out of range");
    if (c->mesh.EToE[size_t(elem[t]) * 4 + face[t]] < 0)
      return c->fail(DG_ERR_ARG, "trace faces must be interior faces");
    for (int m = 0; m < Nfp; ++m) {
      double x[3];
      node_position(c, elem[t], c->ref.Fmask[face[t] * Nfp + m], x);
      for (int d = 0; d < 3; ++d) xyz[(size_t(t) * Nfp + m) * 3 + d] = float(x[d]);
    }
  }
  DG_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c->tr_elem); dfree(c->tr_face); dfree(c->txyz); dfree(c->tr_psi); dfree(c->tr_res);
  c->ntrace = 0;
  if (n == 0) return DG_OK;
  DG_CUDA(cudaMalloc(&c->tr_elem, size_t(n) * 4));
  DG_CUDA(cudaMalloc(&c->tr_face, size_t(n)));
  DG_CUDA(cudaMalloc(&c->txyz, xyz.size() * 4));
  // memories start empty; they also restart with every dg_set_state
  DG_CUDA(cudaMalloc(&c->tr_psi, size_t(n) * Nfp * 4));
  DG_CUDA(cudaMalloc(&c->tr_res, size_t(n) * Nfp * 4));
  DG_CUDA(cudaMemset(c->tr_psi, 0, size_t(n) * Nfp * 4));
  DG_CUDA(cudaMemset(c->tr_res, 0, size_t(n) * Nfp * 4));
  DG_CUDA(cudaMemcpy(c->tr_elem, elem, size_t(n) * 4, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(c->tr_face, face, size_t(n), cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(c->txyz, xyz.data(), xyz.size() * 4, cudaMemcpyHostToDevice));
  c->ntrace = n;
  return DG_OK;
}

int dg_sample_traces(dg_ctx* c, float* X, float* Y, float* amp) {
  if (!c || !X || !Y) return DG_ERR_ARG;
  if (!c->have_state) return c->fail(DG_ERR_ORDER, "no state set");
  if (c->ntrace == 0) return c->fail(DG_ERR_ORDER, "no trace faces set");
  DG_CUDA(dgk::launch_sample_traces(c->q32[c->cur], c->ref.Np, c->ref.Nfp, c->tr_elem, c->tr_face,
                                    c->conn, c->tbl, c->fmask, c->geo32, c->txyz, c->tr_psi,
                                    c->ntrace, base_ghost(c), mlp_scales(c), X, Y, amp, c->status,
                                    c->stream));
  return DG_OK;
}

static int mlp_grad_dev(dg_ctx* c, const float* X, const float* Y, int64_t N) {
  int dev = 0, sms = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int nb = dgk::mlp_grad_blocks(N, sms);
  const size_t need = size_t(nb) * (dgk::mlp::kParams + 1);
  if (need > c->mlp_part_len) {
    dfree(c->mlp_part);
    DG_CUDA(cudaMalloc(&c->mlp_part, need * 4));
    c->mlp_part_len = need;
  }
  DG_CUDA(dgk::launch_mlp_loss_grad(c->mlp_w, X, Y, N, nb, c->mlp_part,
                                    c->mlp_part + size_t(nb) * dgk::mlp::kParams, c->mlp_grad,
                                    c->mlp_loss, c->stream));
  return DG_OK;
}

int dg_mlp_loss_grad(dg_ctx* c, const float* X, const float* Y, int64_t N, double* loss,
                     float* grad) {
  if (!c || !X || !Y || N <= 0) return DG_ERR_ARG;
  if (!c->mlp_w) return c->fail(DG_ERR_ORDER, "no network set");
  int rc = mlp_grad_dev(c, X, Y, N);
  if (rc) return rc;
  DG_CUDA(cudaStreamSynchronize(c->stream));
  if (loss) DG_CUDA(cudaMemcpy(loss, c->mlp_loss, 8, cudaMemcpyDeviceToHost));
  if (grad) DG_CUDA(cudaMemcpy(grad, c->mlp_grad, size_t(dgk::mlp::kParams) * 4, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int dg_mlp_train(dg_ctx* c, const float* X, const float* Y, int64_t N, int iters, double lr,
                 double* loss_history) {
  if (!c || !X || !Y || N <= 0 || iters < 0 || !(lr > 0.0)) return DG_ERR_ARG;
  if (!c->mlp_w) return c->fail(DG_ERR_ORDER, "no network set");
  nvtxRangePushA("dg_mlp_train");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  for (int it = 0; it < iters; ++it) {
    int rc = mlp_grad_dev(c, X, Y, N);
    if (rc) return rc;
    if (loss_history)
      DG_CUDA(cudaMemcpyAsync(loss_history + it, c->mlp_loss, 8, cudaMemcpyDeviceToHost, c->stream));
    ++c->mlp_t;
    DG_CUDA(dgk::launch_adam(c->mlp_w, c->mlp_grad, c->mlp_m, c->mlp_v, float(lr), c->mlp_t, c->stream));
    c->mlp_img_ok = false;
  }
  DG_CUDA(cudaStreamSynchronize(c->stream));
  return DG_OK;
}

int dg_mlp_forward(dg_ctx* c, const float* X, int64_t N, float* out) {
  if (!c || !X || !out || N < 0) return DG_ERR_ARG;
  if (!c->mlp_w) return c->fail(DG_ERR_ORDER, "no network set");
  DG_CUDA(dgk::launch_mlp_forward(c->mlp_w, X, N, out, c->stream));
  return DG_OK;
}

}  // extern "C"
