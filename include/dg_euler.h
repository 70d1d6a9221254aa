/*
 * dg_euler.h - C ABI of the GB300 nodal discontinuous Galerkin solver for the
 * 3D compressible Euler equations on straight-sided tetrahedral meshes with
 * pass-through (non-reflecting) outer boundaries.
 *
 * What is computed (citations are to Resch, "How the three-dimensional
 * geometry of computational domain(s) affects the accuracy of non-reflective
 * boundary conditions in acoustic simulation", arXiv:1710.03887):
 *   - conserved variables (rho, rho u, rho v, rho w, E) of the Euler system,
 *     section 2.1 Eq. 1, closed by the ideal-gas law Eq. 2;
 *   - the element-wise DG semi-discretisation of Appendix A (Eqs. 8-12), in
 *     nodal strong form: dq/dt = -div F + LIFT (Fscale (n.F(q-) - F*));
 *   - local Lax-Friedrichs numerical flux on every face (section 1.1);
 *   - outer-boundary ghost states: the paper's free-stream pass-through
 *     condition (section 2.2), a characteristic (Riemann-invariant)
 *     far-field ghost (section 1), the reflective wall of section 2.3 Eq. 4,
 *     the mouthpiece inflow pulse of section 2.4 (Eqs. 5-7), and a learned
 *     closure (a network trained on the method's own traces, with a
 *     spherical-wave memory after the asymptotic conditions section 1 names);
 *   - time integration of the ODE system of Eq. 12 with the five-stage
 *     2N-storage fourth-order Runge-Kutta scheme of Carpenter & Kennedy (1994);
 *   - sensors (section 3) and the time-integrated boundary flux;
 *   - three arithmetic forms of the time step: float64, a float32
 *     perturbation form, and the float32 form with tensor-core (tcgen05,
 *     TF32x3) contractions.
 *
 * Conventions
 *   - Every function returns an int status: DG_OK (0) or a negative DG_ERR_*.
 *     dg_last_error() gives a message for the last failure on a context.
 *     No C++ exception crosses this interface.
 *   - Host arrays passed in are read during the call and never retained;
 *     arrays passed out are written before the call returns.
 *   - "device" pointers are CUDA global-memory pointers of the current
 *     device (for instance from torch). The library does not retain them.
 *   - The context owns its device buffers (allocated on first device use,
 *     freed by dg_destroy). Device work is enqueued on the stream given by
 *     dg_set_stream (default: the legacy default stream); calls that return
 *     host data synchronise that stream.
 *   - State layout at the interface: q[K][5][Np] (element-major, then
 *     variable, then node), float64, total (not perturbation) state; the
 *     float32 forms convert inside. Node order: lattice (i,j,k), i+j+k <= p, with k
 *     outermost and i innermost; reference tetrahedron vertices v1=(-1,-1,-1),
 *     v2=(1,-1,-1), v3=(-1,1,-1), v4=(-1,-1,1) map to element vertices
 *     EToV[e][0..3].
 *   - A device error (non-finite state, non-positive density or pressure; a
 *     tensor-core completion wait that gave up) is latched in a status word
 *     on the device and reported as DG_ERR_NONFINITE (DG_ERR_TIMEOUT) by the
 *     next call that synchronises (dg_sync, dg_get_state, dg_read_*), which
 *     also clears it; the context stays usable. In the debug build (the same
 *     sources compiled with -DDG_BOUNDS_CHECK into libdgeuler_debug.so) every
 *     index a kernel reads from the mesh tables (face lists, connection
 *     words, node tables, boundary slots, halo rows) is checked before the
 *     access it selects; a failed check skips that access and is reported as
 *     DG_ERR_BOUNDS the same way.
 */
#ifndef DG_EULER_H
#define DG_EULER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_ERR_ARG (-1)         /* bad argument (null pointer, size, range)      */
#define DG_ERR_MESH (-2)        /* inverted element, non-manifold/unmatched face */
#define DG_ERR_CUDA (-3)        /* a CUDA runtime call failed                    */
#define DG_ERR_ORDER (-4)       /* call out of order (e.g. step before state)    */
#define DG_ERR_NONFINITE (-5)   /* device saw a non-finite or non-physical state */
#define DG_ERR_UNSUPPORTED (-6) /* order / mode not built into this library      */
#define DG_ERR_TIMEOUT (-7)     /* a bounded device wait gave up (kernel returned) */
#define DG_ERR_BOUNDS (-8)      /* a device bounds check failed (debug build only)  */

/* dg_build_flags bits */
#define DG_BUILD_BOUNDS_CHECKS 1 /* kernels carry device bounds checks             */

/* Boundary ghost rules (dg_set_bc) */
#define DG_BC_FREESTREAM 0      /* ghost = free-stream state (section 2.2, Eq. 3)       */
#define DG_BC_CHARACTERISTIC 1  /* Riemann-invariant far-field ghost (default)          */
#define DG_BC_SLIP_WALL 2       /* normal velocity mirrored (section 2.3, Eq. 4)        */
#define DG_BC_LEARNED 3         /* characteristic ghost with a learned, bounded incoming */
                                /* invariant (float32 forms; see dg_set_bc_mlp); falls   */
                                /* back to the characteristic ghost where the result is  */
                                /* not finite or has rho <= 0 or p <= 0                  */
#define DG_BC_INFLOW_PULSE 4    /* mouthpiece inflow (section 2.4, Eqs. 5-7): a one-     */
                                /* period pressure pulse entering as a plane wave; see   */
                                /* dg_set_inflow                                         */

/* Arithmetic of the time step (dg_params.precision) */
#define DG_PREC_FP64 0          /* float64 state, fluxes and contractions               */
#define DG_PREC_F32 1           /* float32 perturbation state q - q0 about the resting   */
                                /* free stream (u0 must be 0); fluxes, ghost states      */
                                /* (written without cancellation against p0, c0),        */
                                /* contractions and update in float32; geometry and      */
                                /* operators formed in float64 on the host; the ledger   */
                                /* and totals add in float64. The state still crosses    */
                                /* the ABI as total float64 q[K][5][Np].                 */
#define DG_PREC_F32_TC 2        /* DG_PREC_F32 with both contractions (volume and LIFT,  */
                                /* Eq. 10) as one tcgen05 tensor-core GEMM per tile of   */
                                /* 12 elements, tf32 operands split in head + tail,      */
                                /* float32 accumulation; orders 1..4                     */
#define DG_PREC_MODAL 3         /* the paper's own discretisation (Appendix A): the weak */
                                /* form of Eq. 10 in the orthonormal basis of Eq. 11,    */
                                /* volume integral by a Gauss rule of degree 2p, surface */
                                /* integrals by one of degree 2p+1 (collapsed Gauss-     */
                                /* Jacobi products, one point set per face: the rule of  */
                                /* its lower-numbered element), LLF flux, Heun's second- */
                                /* order Runge-Kutta (section 1.1) in dg_step; float64.  */
                                /* The state crosses the ABI as nodal values of the same */
                                /* polynomials (the nodes of the other forms), so probes,*/
                                /* totals and dg_stable_dt work unchanged.               */
#define DG_PREC_F32_TC1 4       /* DG_PREC_F32_TC with one MMA per k-step: the float32   */
                                /* operands are read as tf32 by the tensor cores (no     */
                                /* head/tail split), so the contractions carry ~2^-10    */
                                /* relative operand error (about 1e-3 of the right-hand  */
                                /* side) against float32's 2^-24: a measured variant of  */
                                /* the contraction's precision, not the float32 form.    */

/* Free-stream gas and defaults of a context. */
typedef struct dg_params {
  double gamma;       /* ratio of specific heats (> 1)                           */
  double rho0;        /* free-stream density (> 0)                                */
  double p0;          /* free-stream pressure (> 0)                               */
  double u0[3];       /* free-stream velocity                                     */
  int32_t default_bc; /* ghost rule of every boundary id until dg_set_bc          */
  int32_t precision;  /* DG_PREC_*                                                */
} dg_params;

typedef struct dg_ctx dg_ctx;

/* Create a solver of polynomial order 1..4 (Np = 4, 10, 20, 35 nodes per
 * element). Builds the reference-element operators on the host (the
 * orthonormal basis of Appendix A, Eq. 11). Touches no GPU. */
int dg_create(int order, const dg_params* params, dg_ctx** out);
/* Free the context and its device buffers (synchronises its stream). NULL ok. */
int dg_destroy(dg_ctx* ctx);
/* Message of the last failed call on ctx (static lifetime within ctx). */
const char* dg_last_error(const dg_ctx* ctx);
/* Stream for all subsequent device work (a cudaStream_t; NULL = default). */
int dg_set_stream(dg_ctx* ctx, void* cuda_stream);

/* Upload a straight-sided tetrahedral mesh (Appendix A, Eq. 9).
 *   xyz[nvert][3]   vertex coordinates
 *   EToV[K][4]      vertex ids per element, positively oriented
 *   face_tag[K][4]  nullable; boundary id 0..7 of faces without a neighbour
 *                   (a negative tag there is an error; tags of interior faces
 *                   are ignored). NULL: every boundary face gets id 0.
 *   vert_class[nvert] nullable; identity used to match faces (vertices with
 *                   equal class are the same vertex for connectivity, e.g. a
 *                   periodic box). NULL: the vertex id itself.
 * Host only: computes J, d(r,s,t)/dx, normals, face areas and connectivity.
 * Errors: DG_ERR_MESH for J <= 0, a face shared by more than two elements,
 * or matched faces that are not back to back. Replaces any previous mesh and
 * invalidates the state. */
int dg_upload_mesh(dg_ctx* ctx, int64_t nvert, const double* xyz, int64_t K,
                   const int32_t* EToV, const int8_t* face_tag,
                   const int64_t* vert_class);
/* A mesh given directly by its geometric factors and connectivity instead
 * of vertices (Appendix A, Eq. 9: the per-element affine maps and the shared
 * faces; e.g. factors computed by another program for parity checks). Host
 * arrays, copied:
 *   drdx[K][3][3]  d r_a / d x_b of element e's affine map (J > 0)
 *   J[K]           determinant of dx/d(r,s,t)
 *   nrm[K][4][3]   outward unit normals of faces 0..3 (t=-1, s=-1,
 *                  r+s+t=-1, r=-1)
 *   Fscale[K][4]   face area / (2 J) (half the area: the surface Jacobian
 *                  over the volume Jacobian)
 *   EToE[K][4]     neighbour element or -1 (boundary face)
 *   EToF[K][4]     neighbour's face (0..3) on interior faces
 *   orient[K][4]   orientation code o (0..5) on interior faces: face vertex c
 *                  of face f of e is face vertex P[o][c] of face EToF of
 *                  EToE, with face f's vertices V[f] = {0,1,2}, {0,1,3},
 *                  {1,2,3}, {0,2,3} (element vertices in the order of the
 *                  affine map) and P = {0,1,2}, {0,2,1}, {1,0,2}, {1,2,0},
 *                  {2,0,1}, {2,1,0}
 *   bc[K][4]       boundary id (0..7) on boundary faces (nullable: 0)
 * Errors (DG_ERR_MESH): J <= 0, normals not of unit length, Fscale <= 0,
 * neighbour links that are not mutual, orientation codes that are not
 * inverse permutations of each other, interior normals not back to back.
 * Without vertex coordinates, dg_node_coords, dg_set_probes, the learned
 * closure and trace recording report DG_ERR_ORDER. Replaces any previous
 * mesh and invalidates the state. */
int dg_upload_geometry(dg_ctx* ctx, int64_t K, const double* drdx, const double* J,
                       const double* nrm, const double* Fscale, const int32_t* EToE,
                       const int8_t* EToF, const int8_t* orient, const int8_t* bc);
/* Ghost rule of boundary id bc_id (0..7). */
int dg_set_bc(dg_ctx* ctx, int bc_id, int mode);
/* Inflow pulse of DG_BC_INFLOW_PULSE (section 2.4): at stage time t the ghost
 * is p = p0 (1 + A (1 - cos(alpha t))) while 0 <= t < 2 pi / alpha (p0
 * afterwards), rho = rho0 (p/p0)^(1/gamma) (Eq. 6), velocity
 * (p - p0)/(rho0 c0) along the inward normal (Eq. 5; the paper's bore axis),
 * E from Eq. 2. The paper's pulse is A = 0.05 (a 10 % p0 peak) with
 * alpha = 565 in its time unit (the defaults). DG_ERR_ARG unless alpha > 0
 * and A > -1/2. */
int dg_set_inflow(dg_ctx* ctx, double amplitude, double alpha);
/* Sizes: number of elements, nodes per element, nodes per face. */
int dg_sizes(const dg_ctx* ctx, int64_t* K, int32_t* Np, int32_t* Nfp);
/* Physical node coordinates xyz[K][Np][3] (host). */
int dg_node_coords(const dg_ctx* ctx, double* xyz);
/* Geometric factors as computed by dg_upload_mesh (host; any pointer may be
 * NULL): J[K], drdx[K][3][3] (d r_a / d x_b), nrm[K][4][3], sJ[K][4],
 * EToE[K][4] (-1 on boundary faces), EToF[K][4], bc[K][4] (-1 interior). */
int dg_get_geometry(const dg_ctx* ctx, double* J, double* drdx, double* nrm,
                    double* sJ, int32_t* EToE, int8_t* EToF, int8_t* bc);
/* Face-node pairing the stage kernels use (host; either pointer may be
 * NULL). Neighbours couple only through the numerical flux at the points of
 * their shared face (section 1.1, the surface term of Eq. 10); the kernels
 * find the other side's value at face node m of face f of element e from
 * the face's connection word (neighbour e2, its face f2, orientation code)
 * and the reference face-node tables. Decoded the same way here:
 * vol_node[K][4][Nfp] = e2 * Np + n2, the neighbour's volume node at that
 * point, and face_node[K][4][Nfp] = the position of n2 in face f2's node
 * list; both -1 on boundary faces. DG_ERR_ORDER before a mesh upload. */
int dg_face_pairs(const dg_ctx* ctx, int64_t* vol_node, int32_t* face_node);
/* Stable time step  cfl * min_e r_in / ((p+1)^2 * max(|u| + c))  of a host
 * state q[K][5][Np] (host computation; r_in = 3 V / total face area). */
int dg_stable_dt(const dg_ctx* ctx, const double* q, double cfl, double* dt);

/* Reference operators of order p (host only, no context): node coordinates
 * rst[3][Np], derivative matrices Dr/Ds/Dt[Np][Np] (row = node where the
 * derivative is taken), LIFT[Np][4*Nfp], Fmask[4][Nfp]. Any output may be
 * NULL. */
int dg_reference_operators(int order, double* rst, double* Dr, double* Ds,
                           double* Dt, double* LIFT, int32_t* Fmask);

/* Gauss rules of DG_PREC_MODAL at order 1..4 (host only, no context):
 * vol[Nq][4] = (r, s, t, weight) on the reference tetrahedron, exact to
 * degree 2p; face[Nfq][3] = (u, v, weight) on the triangle (-1,-1), (1,-1),
 * (-1,1), exact to degree 2p+1; Nq = (p+1)^3, Nfq = (p+1)^2 (Appendix A's
 * 2p / 2p+1 rules as collapsed Gauss-Jacobi products). Either array may be
 * NULL; nq/nfq (nullable) receive the counts. */
int dg_modal_quadrature(int order, double* vol, double* face, int32_t* nq, int32_t* nfq);
/* Operators of DG_PREC_MODAL on nodal values (host only, no context), with
 * Nq, Nfq as above (Appendix A's weak form, Eq. 10, in the orthonormal
 * basis, Eq. 11):
 *   du_n/dt = sum_a sum_q Sv[a][n][q] G_a(x_q) - sum_f Fscale_f sum_q Sf[f][v_f][n][q] F*_q
 * Iq[Nq][Np]: nodal values -> volume points; Sv[3][Np][Nq]; Ifn[4][7][Nfq][Nfp]:
 * face-node values (Fmask order) -> face points; Sf[4][7][Np][Nfq]; wf[Nfq]
 * face weights. Face variant v_f = 0 when the element's index is not above
 * its neighbour's (and on outer faces), else 1 + the face's orientation
 * code. Any output may be NULL. */
int dg_modal_operators(int order, double* Iq, double* Sv, double* Ifn, double* Sf, double* wf);

/* State q[K][5][Np] from host memory at time t; resets the Runge-Kutta
 * residual, the boundary-flux ledger and the probe buffer. */
int dg_set_state(dg_ctx* ctx, const double* q, double t);
/* Same, from a device pointer. */
int dg_set_state_device(dg_ctx* ctx, const double* dq, double t);
/* Copy the state to host memory (synchronises); t may be NULL. */
int dg_get_state(dg_ctx* ctx, double* q, double* t);
/* Copy the state to a device buffer (enqueued on the stream; t on host). */
int dg_get_state_device(dg_ctx* ctx, double* dq, double* t);

/* Advance n full time steps of size dt (n >= 0, dt > 0): 5 Runge-Kutta stages
 * each, every stage one evaluation of the semi-discrete operator (Eq. 12).
 * Enqueued on the stream; returns without waiting. */
int dg_step(dg_ctx* ctx, int n, double dt);
/* One evaluation of the right-hand side f(q) of Eq. 12 at the current state
 * and time, copied to host rhs[K][5][Np] (synchronises). Does not change the
 * state or the time-stepping residual. */
int dg_eval_rhs(dg_ctx* ctx, double* rhs);

/* Sensors (section 3): n points xyz[n][3], each located in the element of
 * lowest index that contains it (barycentrics >= -1e-12); DG_ERR_ARG if a
 * point lies outside the mesh. After every completed step the five conserved
 * variables are interpolated at each point into a device ring buffer of
 * `capacity` steps. */
int dg_set_probes(dg_ctx* ctx, int n, const double* xyz, int capacity);
/* Read the samples recorded since the last read, oldest first, as
 * out[steps][n][5] (host); at most min(max_steps, capacity) steps, the most
 * recent ones if more were recorded. *got = steps written. Synchronises. */
int dg_read_probes(dg_ctx* ctx, int max_steps, double* out, int* got);

/* Time integral, since dg_set_state, of the outward numerical flux through
 * all boundary faces: out[5] (host, synchronises). With it,
 * totals(t) - totals(0) + ledger(t) = 0 up to rounding. */
int dg_read_boundary_flux(dg_ctx* ctx, double out[5]);
/* Conserved totals  sum_e J_e 1^T M q_e  (host, synchronises). */
int dg_conserved_totals(dg_ctx* ctx, double out[5]);

/* Wait for the stream; report (and clear) a latched device error. */
int dg_sync(dg_ctx* ctx);

/* Build of the loaded library (no counterpart in the paper: a checking aid).
 * *flags = DG_BUILD_BOUNDS_CHECKS for the debug build, 0 for the release
 * build. DG_ERR_ARG for a null pointer. */
int dg_build_flags(int* flags);
/* Debug build only (no counterpart in the paper): one device thread fails a
 * bounds check on purpose, with no out-of-range access, so a caller can see
 * a failed check reach it: the next synchronising call returns
 * DG_ERR_BOUNDS. Needs an uploaded mesh (DG_ERR_ORDER otherwise);
 * DG_ERR_UNSUPPORTED in the release build. */
int dg_bounds_selftest(dg_ctx* ctx);

/* Per-launch timing of the Runge-Kutta stage kernel: when enabled, dg_step
 * records a CUDA event pair on the stream around every stage launch.
 * dg_read_kernel_timing synchronises, returns the summed stage-kernel time in
 * milliseconds and the number of timed launches since the last read, and
 * resets both. Enabling/disabling discards pending records. */
int dg_set_kernel_timing(dg_ctx* ctx, int enable);
int dg_read_kernel_timing(dg_ctx* ctx, double* total_ms, int64_t* launches);

/* ------------------------------------------------------------------------
 * Learned boundary closure (boundary mode DG_BC_LEARNED, float32 forms). The
 * paper's pass-through condition (section 2.2) and the characteristic ghost
 * both assume what lies outside the truncation surface; section 1 names the
 * asymptotic far-field conditions as the other route. This closure starts
 * from the lowest-order such condition for an outgoing spherical wave and
 * learns the rest from the method's own solution in a larger domain.
 *
 * At every node of an outer face with this mode, with perturbation trace
 * q' = q- - q0 (rho', m', E'), rho = rho0 + rho', u = m'/rho,
 * p' = (gamma - 1)(E' - |m'|^2 / (2 rho)), outward unit normal n, node
 * position x, scale R (dg_set_bc_mlp), c0^2 = gamma p0 / rho0, Z = rho0 c0:
 *   w_out = p' + Z u.n          outgoing acoustic invariant of the trace
 *   psi   memory of the node: d psi/dt = -(c0 / (2 r)) (psi + w_out),
 *         r = max(|x|, 1e-3 R), advanced by the same Runge-Kutta stages as
 *         the state, zero after dg_set_state. For an outgoing spherical wave
 *         of linear acoustics centred at the origin, psi is exactly the
 *         incoming invariant.
 *   s     = (|w_out| + |psi|) / (rho0 c0^2) + 1e-12   (amplitude)
 *   features f[12] = ( w_out / (rho0 c0^2 s),
 *                      (rho' - p'/c0^2) / (rho0 s),
 *                      u_t / (c0 s)  (3; u_t = u - (u.n) n),
 *                      n  (3),
 *                      x / R  (3),
 *                      psi / (rho0 c0^2 s) )
 * A network 12 -> 64 -> 64 -> 5 (tanh hidden layers, linear output, float32)
 * maps f to y; only y[0] is used (outputs 1..4 are trained towards zero).
 * The ghost's incoming invariant is
 *   g = clamp(psi + rho0 c0^2 s y[0], -L, L),  L = max(|w_in,c|, rho0 c0^2 s),
 * with w_in,c = p'_c - Z u_c.n the incoming invariant of the characteristic
 * ghost of the same trace. The ghost is that characteristic ghost moved along
 * the incoming acoustic wave by D = g - w_in,c:
 *   rho += D / (2 c0^2),  m -= D n / (2 c0),  E += D / (2 (gamma - 1)).
 * The characteristic ghost is kept where the result is not finite or has
 * rho <= 0 or p <= 0, and on every node while no parameters are set. An
 * all-zero output layer (y = 0) gives g = psi, the spherical-wave condition;
 * since |psi| <= rho0 c0^2 s <= L the bound never cuts that value. The bound
 * limits |g| only; it is not an energy or stability guarantee.
 *
 * Worked example (rho0 = 1, gamma = 1.4, p0 = 1/1.4, so c0 = 1): the trace
 *   q' = (0.01, 0.02, -0.03, 0.04, 0.05), n = (0, 0, 1), x = (0.3, -0.4, 1.2),
 *   R = 2, psi = -0.02
 * has w_out = 0.0590297030, s = 0.0790297030 (+1e-12) and features
 * EXAMPLE_FEATURES: 0.7469305938 -0.1192683538 0.2505637685 -0.3758456527 0 0 0 1 0.15 -0.2 0.6 -0.2530694062
 *
 * Parameters (DG_MLP_NPARAMS floats, row-major, input index first):
 *   W1[12][64], b1[64], W2[64][64], b2[64], W3[64][5], b3[5];
 *   y = tanh(tanh(f W1 + b1) W2 + b2) W3 + b3.
 * Training minimises (1/N) sum |network(features) - target|^2 over samples
 * recorded with dg_sample_traces, full batch, Adam (beta 0.9 / 0.999,
 * eps 1e-8), on the GPU. All float32. */
#define DG_MLP_NPARAMS 5317

/* Mass matrix M[Np][Np] of the reference element (host only, no context). */
int dg_reference_mass(int order, double* M);
/* Set the network parameters (host array of DG_MLP_NPARAMS floats) and the
 * position scale R; resets the optimiser state. Allocates on first use. */
int dg_set_bc_mlp(dg_ctx* ctx, const float* w, double radius);
/* Copy the current network parameters to host memory. */
int dg_get_bc_mlp(dg_ctx* ctx, float* w);
/* Interior faces at which dg_sample_traces records (float32 forms only):
 * face face[i] (0..3) of element elem[i], whose element is the inside.
 * DG_ERR_ARG for boundary faces or ids out of range. */
int dg_set_trace_faces(dg_ctx* ctx, int64_t n, const int32_t* elem, const int8_t* face);
/* Training pairs from the current state at every node of the trace faces:
 * X[n*Nfp][12] the features above of the inner trace and its memory,
 * Y[n*Nfp][5] the target output: Y0 = (w_in(outer trace) - psi) /
 * (rho0 c0^2 s), what the outer trace's incoming invariant adds to the
 * memory's spherical-wave value, Y1..4 = 0; amp[n*Nfp] (nullable)
 * the amplitude rho0 c0^2 s = |w_out| + |psi| in pressure units, for choosing
 * the samples a wave has reached. The memories of the trace nodes restart at
 * zero with dg_set_state and advance with every dg_step.
 * X, Y, amp: device float32 buffers (caller-owned); enqueued on the stream. */
int dg_sample_traces(dg_ctx* ctx, float* X, float* Y, float* amp);
/* Loss and gradient of the current network on device samples X[N][12],
 * Y[N][5] (deterministic fixed-order reductions); either output may be NULL
 * (host, double loss, float gradient[DG_MLP_NPARAMS]). Synchronises. */
int dg_mlp_loss_grad(dg_ctx* ctx, const float* X, const float* Y, int64_t N, double* loss,
                     float* grad);
/* `iters` full-batch Adam steps with learning rate lr on device samples;
 * loss_history (host, nullable) receives the loss before each step. */
int dg_mlp_train(dg_ctx* ctx, const float* X, const float* Y, int64_t N, int iters, double lr,
                 double* loss_history);
/* Network outputs out[N][5] (device) for features X[N][12] (device). */
int dg_mlp_forward(dg_ctx* ctx, const float* X, int64_t N, float* out);

/* ------------------------------------------------------------------------
 * Partitioned meshes (one rank per GPU). The element partition of Omega
 * (Appendix A, Eq. 9) lets each rank own a set of elements; a face between
 * elements of two ranks (a cut face) needs, once per Runge-Kutta stage, the
 * neighbour's trace on that face (the surface term of Eq. 10). A rank's mesh
 * holds its own elements first, then copies of the neighbour elements
 * across its cut faces (halo elements); faces of a halo element that lead
 * nowhere on this rank carry any boundary id (they are never evaluated).
 *
 * dg_set_owned: elements [0, K_own) are this rank's, [K_own, K) halo copies.
 *   Halo elements are never advanced; totals, the boundary ledger and
 *   sensors count own elements only (a sensor must lie in an own element).
 *   Call after the mesh upload and before dg_set_state (it discards device
 *   buffers). DG_ERR_UNSUPPORTED for DG_PREC_MODAL: the paper's
 *   discretisation picks each face's quadrature points by element number,
 *   which a partition renumbers.
 * dg_set_halo: the exchange lists (host arrays, copied): send entry i is
 *   face send_face[i] of own element send_elem[i] (a cut face); receive entry
 *   i is face recv_face[i] of halo element recv_elem[i] (its face to an own
 *   element). DG_ERR_ARG for an entry that is not such a face. Call after
 *   dg_set_owned.
 * dg_halo_pack: buf[n_send][5][Nfp] <- the current state at the nodes of the
 *   send faces (face node order of the reference element), in the state's
 *   own representation: double total state for DG_PREC_FP64, float
 *   perturbation q - q0 for the float32 forms. Device buffer, caller-owned,
 *   enqueued on the stream.
 * dg_halo_unpack: the current state at the nodes of the receive faces <-
 *   buf[n_recv][5][Nfp] (same layout and type). A receive entry's buffer row
 *   is the send row of the same face on the rank that owns the element.
 * dg_step_stages: advance n Runge-Kutta stages (continuing a step in
 *   progress); the time advances and the sensors sample after the last stage
 *   of a step. A partitioned run exchanges halos before every stage:
 *   pack, send / receive, unpack, dg_step_stages(1). dg_step refuses
 *   (DG_ERR_ORDER) while a step is in progress; dg_set_state ends it.
 * dg_stage_index: the next stage (0..stages_per_step - 1) and the stages per
 *   step (5 for the Runge-Kutta forms, 2 for the paper's Heun scheme). */
int dg_set_owned(dg_ctx* ctx, int64_t K_own);
int dg_set_halo(dg_ctx* ctx, int64_t n_send, const int32_t* send_elem, const int8_t* send_face,
                int64_t n_recv, const int32_t* recv_elem, const int8_t* recv_face);
int dg_halo_pack(dg_ctx* ctx, void* buf);
int dg_halo_unpack(dg_ctx* ctx, const void* buf);
int dg_step_stages(dg_ctx* ctx, int n, double dt);
int dg_stage_index(dg_ctx* ctx, int* k, int* stages_per_step);

/* Conserved totals that allocate nothing (no counterpart in the paper: this
 * is a service for callers that cannot call cudaMalloc where they need the
 * totals, e.g. code whose device memory is entirely owned by another
 * allocator, or monitoring code inside a running time loop that must not
 * allocate or free device memory).
 *   out[v] = sum_e J[e] sum_i w[i] q[e][v][i],  v = 0..4
 * q[K][5][Np], J[K], w[Np] (the mass-matrix column sums 1^T M of the
 * reference element) and out[5] are device pointers supplied and owned by
 * the caller; work is enqueued on `stream` (a cudaStream_t, NULL = default)
 * and the call returns without waiting. The per-block partial sums live in
 * one file-scope device array of DG_STATIC_TOTALS_MAX_BLOCKS x 5 doubles
 * (160 KiB), which every GPU that loads the library keeps until the process
 * exits. The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture. The address is kept per device and context: the
 * first call after a cudaDeviceReset looks it up again and is a first call in
 * that sense. Errors are those of this call's own launches (an earlier
 * asynchronous error on the thread is left for the caller to read). All calls share the array and it keeps the last
 * call's contents (nothing in it needs to start at zero); calls on the same
 * device that can overlap on the GPU (for instance on different streams)
 * race on the array and must be serialised by the caller. Returns DG_ERR_ARG for a null pointer, K <= 0,
 * K > DG_STATIC_TOTALS_MAX_ELEMENTS or Np outside 1..DG_STATIC_TOTALS_MAX_NP,
 * before touching any memory. */
#define DG_STATIC_TOTALS_MAX_BLOCKS 4096
#define DG_STATIC_TOTALS_ELEMS_PER_BLOCK 4096
#define DG_STATIC_TOTALS_MAX_ELEMENTS (4096LL * 4096LL)
#define DG_STATIC_TOTALS_MAX_NP 35
int dg_weighted_totals_static(const double* q, const double* J, const double* w,
                              int64_t K, int Np, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DG_EULER_H */
