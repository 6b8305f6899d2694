/*
 * demag.h -- C ABI of libdemag: the demagnetizing (scalar potential) operator
 * of arXiv 1212.3509 (Exl, Abert, Mauser, Schrefl, Stimming, Suess, "FFT-based
 * Kronecker product approximation to micromagnetic long-range interactions")
 * applied as a sum of Kronecker products on one GB300 GPU (sm_103a).
 *
 * What is computed (paper Sec. 3, Eq. coll, Eq. pot_op, Cor. 3 Eq. kron_operator):
 *
 *   phi_i = c * s * sum_{k=1..M} omega_k sum_{q=1..3} sum_j
 *                 T_{k,q,3}[i3-j3] T_{k,q,2}[i2-j2] T_{k,q,1}[i1-j1] m^(q)_j
 *
 *   c = 1/(2 pi^{3/2}),  T_{k,q,p} = F_k^(p) if p == q else E_k^(p),
 *   E_k^(p)[d] = int_{(d-1/2)h}^{(d+1/2)h} exp(-tau_k^2 x^2) dx,
 *   F_k^(p)[d] = int_{(d-1/2)h}^{(d+1/2)h} x exp(-tau_k^2 x^2) dx   (Eq. f_anal),
 *   tau_k = sinh(k theta), omega_k = 2 theta cosh(k theta) sinh(k theta)^2,
 *   theta = c0 ln(M)/M, R = 2M+1 symmetric sinc nodes (Thm. 1, Lemma 2).
 *
 * Conventions used by every entry point:
 *  - Units: reduced (|m| = 1).  The domain is scaled so that its longest edge
 *    is 1 before the nodes are applied (Sec. 3.4, rho <= 3); s = max_p n_p h_p
 *    and hh_p = h_p / s are used for the generators and phi is returned in the
 *    caller's length unit (multiplied by s).
 *  - Sign: phi = +(1/4pi) int m.(x-y)/|x-y|^3, the sign that solves
 *    Delta phi = div m with h_d = -grad phi (Eq. poisson, Eq. intop1); the
 *    printed Eq. intop2 / coll / kron_operator carry the opposite sign.
 *  - Layout: a scalar field is float [n3][n2][n1] (i1 fastest, the vec order of
 *    the footnote to Cor. 3); a magnetization is float [3][n3][n2][n1].
 *  - Memory: every data pointer is a DEVICE pointer owned by the caller; the
 *    library never frees or retains it after the call returns.  The plan owns
 *    its generators, symbols, dense factor matrices and workspace.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *    compute entry points are asynchronous on that stream, except the
 *    host-driven ones documented as synchronous (kernel compression,
 *    recompression, TT rounding).
 *  - Errors: arguments are validated before any launch; a rejected call
 *    returns DEMAG_EINVAL (or DEMAG_EUNSUPPORTED) and launches nothing.  A
 *    failed launch returns DEMAG_ECUDA.  The message of the last error of a
 *    plan is returned by demag_last_error (plan may be NULL for errors raised
 *    before a plan exists).  No entry point aborts the process.
 *  - Threads: a plan must not be used from two host threads at once.
 */
#ifndef DEMAG_H
#define DEMAG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DEMAG_OK = 0,
  DEMAG_EINVAL = 1,      /* bad argument (NULL pointer, size, rank, R, c0) */
  DEMAG_ENOMEM = 2,      /* device allocation failed */
  DEMAG_ECUDA = 3,       /* a CUDA runtime call or launch failed */
  DEMAG_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
  DEMAG_EUNSUPPORTED = 5 /* valid request outside the library's limits */
} demag_status;

/* Arithmetic of the full-format mode products (Sec. 2.2 Eq. modemul).
 * FP64 / FP32: SIMT (CUDA cores).  TF32X3 / BF16X3: tcgen05 tensor cores with
 * each operand split into a high and a low part and three products
 * (hi*hi + hi*lo + lo*hi) accumulated in FP32. */
typedef enum {
  DEMAG_FP64 = 0,
  DEMAG_FP32 = 1,
  DEMAG_TF32X3 = 2,
  DEMAG_BF16X3 = 3
} demag_precision;

/* Grid and quadrature (Sec. 3.1 notation; Alg. 2 signature potential(M, h, R, c0, tol)).
 * n[p] >= 1 cells on axis p (n[0] = n1 is the fastest index), h[p] > 0 the
 * cell edge, R = 2M+1 odd, 5 <= R <= 513 (M <= 256), the number of symmetric
 * sinc nodes (the rule is not uniform in h, Remark after Lemma 2: R grows with
 * n), c0 > 0 the step constant (2.15 in Sec. 3.4, Fig. 1).  Larger R is
 * rejected with DEMAG_EUNSUPPORTED; demag_compress_kernel takes R <= 129. */
typedef struct {
  int n[3];
  double h[3];
  int R;
  double c0;
} demag_grid_desc;

typedef struct demag_plan demag_plan;

/* ---- setup -------------------------------------------------------------- */

/* Build a plan: sinc nodes, FP64 generators E_k^(p), F_k^(p) (Eq. f_anal,
 * erfc/erfcx/expm1 forms), their FP32 copies, the circulant symbols of the
 * structured path (Sec. 4.2 Eq. conv_pot / fft_pot: real FFT of the length
 * L_p = pow2 >= 2 n_p - 1 embedding, computed in FP64) and the dense Toeplitz
 * factor matrices of the full path (Cor. 3, U_k^(qp)).  Setup is done once
 * per grid (Sec. 4.2: the kernel is built in a setup phase).  Allocates
 * device memory and synchronizes `stream` before returning.
 * On success *out receives the plan; on failure *out is set to NULL. */
demag_status demag_build_factors(const demag_grid_desc* desc, demag_plan** out, void* stream);

/* A non-uniform tensor grid (Sec. 3.1 notation: each axis partitioned into
 * arbitrary sub-intervals I_j = [edges[p][j], edges[p][j+1]], collocation at
 * their midpoints).  edges[p] points to n[p] + 1 strictly increasing finite
 * doubles in HOST memory, read only during the build; n[0] is the fastest
 * index as in demag_grid_desc. */
typedef struct {
  int n[3];
  const double* edges[3];
  int R;
  double c0;
} demag_grid_edges_desc;

/* Build a plan for a non-uniform tensor grid.  The factors of Eq. sep_integrands
 * are then dense n_p x n_p matrices (cell integrals with the true limits, FP64,
 * the same erf/erfcx/expm1 forms as the uniform generators), no longer Toeplitz,
 * and the domain is scaled by its longest edge as in the uniform case.  Such a
 * plan serves the full format: demag_apply_full in all four precisions
 * (batched and graph forms included) and demag_apply_adjoint in DEMAG_FP32 and
 * DEMAG_FP64 (transposed factors: P^T = -P holds only on uniform grids).  Every
 * path that needs Toeplitz structure or uniform spacing (CP / Tucker / TT, the
 * 3D FFT convolution, the finite-difference stray field and energy, the
 * analytic stray field, the split-precision adjoint, generator and symbol
 * copies) returns DEMAG_EUNSUPPORTED for it.  Synchronizes `stream`. */
demag_status demag_build_factors_nonuniform(const demag_grid_edges_desc* desc, demag_plan** out,
                                            void* stream);

/* Release every device buffer the plan owns.  NULL is accepted. */
void demag_plan_destroy(demag_plan* plan);

/* Number of folded quadrature terms M = (R-1)/2 (the term count of every
 * structured output), or -1 for a NULL plan. */
int demag_num_terms(const demag_plan* plan);

/* Text of the last error recorded on `plan` (or of the last error of a call
 * made without a plan when plan == NULL).  Never NULL. */
const char* demag_last_error(const demag_plan* plan);

/* Copy the setup data to caller device buffers (for verification):
 * nodes: double [3][M] = t_k, tau_k, omega_k;  generators: double
 * [M][2][3][2*nmax-1], type 0 = E, 1 = F, entry d + n_p - 1 for
 * d = -(n_p-1)..n_p-1 (unused tail entries of short axes are 0);
 * symbols: float [M][2][3][Lmax/2+1], the real FFT of the circulant
 * embedding divided by L_p (E: real part, F: imaginary part; the other part
 * is 0 by symmetry).  Synchronous on `stream`. */
demag_status demag_copy_nodes(const demag_plan* plan, double* dst, void* stream);
demag_status demag_copy_generators(const demag_plan* plan, double* dst, void* stream);
demag_status demag_copy_symbols(const demag_plan* plan, float* dst, void* stream);
/* Sizes in elements of the three buffers above. */
size_t demag_generators_size(const demag_plan* plan);
size_t demag_symbols_size(const demag_plan* plan);

/* ---- full format (Cor. 3, Eq. kron_operator; Sec. 2.2 Eq. modemul) -------- */

/* phi = sum_q P^(q) m^(q) for a full magnetization.
 * m: float [3][n3][n2][n1], phi: float [n3][n2][n1] (overwritten).
 * Per node the nine mode products share work: 8 GEMMs of n^4 flops-pairs
 * (mode 1: F m1, E m2, E m3; mode 2: E Y1 + F Y2, E Y3; mode 3 with the node
 * sum folded into the contraction).  The first call of a precision allocates
 * its workspace (so make it before any stream capture).  m and phi must not
 * overlap. */
demag_status demag_apply_full(demag_plan* plan, const float* m, float* phi,
                              demag_precision prec, void* stream);

/* The same phi = sum_q P^(q) m^(q) by one 3D FFT convolution (Sec. 4.2,
 * Eq. conv_pot and Eq. fft_pot): the node sum is folded once per plan into a
 * dense Fourier kernel K^(q) on the padded grid L_p (the plan's power of two
 * >= 2 n_p - 1), so an application costs five passes of FP32 shared-memory
 * FFTs independent of R.  m: float [3][n3][n2][n1], phi: float [n3][n2][n1]
 * (overwritten), device pointers, 4-byte aligned, not overlapping.  The
 * first call builds the kernel (FP64 sums, stored FP32: 12 (L1/2+1)
 * (L2/2+1) (L3/2+1) bytes) and the spectra workspace (about
 * 8 (3 (L1/2+1) n3 n2 + 3 L2 (L1/2+1) n3) bytes), so make it before any
 * stream capture; later calls allocate nothing.  Asynchronous on `stream`.
 * DEMAG_EUNSUPPORTED when some n_p > 1024. */
demag_status demag_apply_full_fft(demag_plan* plan, const float* m, float* phi, void* stream);

/* The same phi by per-fibre 1D Toeplitz FFTs (Sec. 4.2 applied to the mode
 * products of Eq. kron_operator, O(R n^3 log n)): the axis-1 fibres of each
 * component through the circulant FFT kernel for all M nodes at once, then
 * the axis-2 and axis-3 fibres of every (node, component) volume with that
 * node's factor, batched transposes between the stages, and the weighted sum
 * over nodes and components.  FP32.  m: float [3][n3][n2][n1], phi: float
 * [n3][n2][n1] (overwritten), device pointers, not overlapping.  The first
 * call allocates two work volumes of 3 M n1 n2 n3 floats each in the plan
 * (make it before any stream capture).  Asynchronous on `stream`.
 * DEMAG_EUNSUPPORTED when some n_p exceeds the FFT path's length. */
demag_status demag_apply_full_fibres(demag_plan* plan, const float* m, float* phi, void* stream);

/* The stray field h_d = -grad phi of demag_stray_field_exact (analytic
 * derivative factors, h_d[p] = sum_q K_pq * m^(q)) by one 3D FFT convolution:
 * the six node-summed derivative kernels K_pq (real, K_pq = K_qp) are built
 * once per plan (FP64 sums, stored FP32 on the octant: 24 prod_p (L_p/2+1)
 * bytes) and an application is five FFT passes, the axis-3 pass multiplying
 * the three component spectra by the 3 x 3 kernel.  m: float [3][n3][n2][n1],
 * hd: float [3][n3][n2][n1] (overwritten), device pointers, not overlapping.
 * The first call builds the kernels and grows the spectra workspace (make it
 * before any stream capture).  Uniform grids with n_p <= 1024 only
 * (DEMAG_EUNSUPPORTED otherwise).  Asynchronous on `stream`. */
demag_status demag_stray_field_fft(demag_plan* plan, const float* m, float* hd, void* stream);

/* Demag energy from the analytic stray field of demag_stray_field_fft:
 * E = -1/2 h1 h2 h3 sum_i m_i . h_d,i (FP64 sum) and, when grad is not NULL,
 * dE/dm = -h1 h2 h3 h_d (the field operator is symmetric: its Fourier kernels
 * are real with K_pq = K_qp, so its real-space kernels are even).  energy: one
 * double on the device (overwritten); grad: float [3][n3][n2][n1].  Uses a
 * plan-owned field buffer (3 fields, allocated on the first call).  This is
 * the energy of the analytic collocation field; demag_energy uses the
 * second-order difference field instead. */
demag_status demag_energy_field_fft(demag_plan* plan, const float* m, double* energy, float* grad, void* stream);

/* Apply several plans' operators in one call: phi[i] = P_i m[i] for
 * i < count.  Arrays of device pointers live in HOST memory.  Grids may
 * differ in shape; every plan must already have its workspace for `prec`
 * (made by a previous demag_apply_full or demag_reserve_workspace).
 * With DEMAG_TF32X3 / DEMAG_BF16X3 a group of listed grids runs as one split
 * launch, one fused mode-1 / mode-2 launch over the grids whose forward
 * schedule is the fused one (demag_forward_schedule; absent when none is),
 * ONE persistent tensor-core launch for every remaining mode-product stage of
 * every grid (tiles of every grid drawn from one work counter, later stages
 * of a grid waiting for its earlier ones), one CUDA-core launch for the last
 * stages along a short third axis (at most 16 cells, films), and one
 * reduction launch; every tile runs the MMA sequence of the grid's own call
 * and a short last stage the same CUDA-core kernel, so a grid whose first two
 * axes are longer than 16 cells gets the bits of demag_apply_full (a short
 * first or second axis runs as padded tensor-core tiles in the batch).  A plan listed twice starts a
 * second such group after the first.  Device-side errors of a group are reported on its
 * first plan (demag_sync_status).  The grouped descriptors are cached on the
 * first plan for the last list seen; the first call with a new list
 * allocates them. */
demag_status demag_apply_full_batched(demag_plan* const* plans, const float* const* m,
                                      float* const* phi, int count, demag_precision prec,
                                      void* stream);

/* ---- CUDA-graph form of the batched apply --------------------------------
 * demag_graph_create_batched records everything demag_apply_full_batched
 * would launch for these plans and pointers into a CUDA graph (captured on a
 * stream of the library's own, nothing runs), instantiates it and returns a
 * handle; demag_graph_launch replays it on `stream`.  The plans must be
 * distinct, have their workspace for `prec`, and outlive the graph; the
 * pointers m[i], phi[i] are baked in (update the buffers, not the pointers).
 * Replays of one graph, and calls on the same plans, must not overlap in
 * time (they share the plans' intermediates).  Kernel-family profiling
 * (demag_profile) does not see graph replays. */
typedef struct demag_graph demag_graph;
demag_status demag_graph_create_batched(demag_plan* const* plans, const float* const* m,
                                        float* const* phi, int count, demag_precision prec,
                                        demag_graph** out);
demag_status demag_graph_launch(demag_graph* graph, void* stream);
/* Kernels one replay launches (the graph's kernel nodes). */
int demag_graph_kernel_count(const demag_graph* graph);
void demag_graph_destroy(demag_graph* graph);

/* Allocate the full-format workspace of `prec` now (idempotent). */
demag_status demag_reserve_workspace(demag_plan* plan, demag_precision prec);

/* Adjoint: g^(q) = (P^(q))^T y for q = 1..3.  E is even and F odd in d (Sec.
 * 4.2), so each transposed Kronecker term equals minus the term itself; the
 * map is one field in, three fields out.  y: float [n3][n2][n1],
 * g: float [3][n3][n2][n1] (overwritten). */
demag_status demag_apply_adjoint(demag_plan* plan, const float* y, float* g,
                                 demag_precision prec, void* stream);

/* ---- structured formats through circulant FFTs (Sec. 4, Lemmas 4-5) ----- */

/* CP input (Eq. CP, one CP tensor per component q) -> CP output
 * (Eq. kron_eval_cp): term (k, q, l) has weight c s omega_k lambda[q][l] and
 * factor columns T_{k,q,p} u^(q,p)_l, p = 1..3.  Every Toeplitz matvec runs as
 * a zero-padded real FFT of length L_p, a product with the symbol and an
 * inverse real FFT keeping the first n_p entries.
 * lambda: float [3][r]; U: float, blocks (q, p) in order q-major, each block
 * [r][n_p] (a column is contiguous); out_w: float [M][3][r];
 * out_U: float, three mode blocks p = 1..3, block p = [M][3][r][n_p].
 * r >= 1. */
demag_status demag_apply_cp(demag_plan* plan, int r, const float* lambda, const float* U,
                            float* out_w, float* out_U, void* stream);

/* `batch` independent CP inputs in one launch: input b starts at
 * lambda + b*3*r and U + b*3*r*(n1+n2+n3); output b at out_w + b*M*3*r and
 * out_U + b*M*3*r*(n1+n2+n3). */
demag_status demag_apply_cp_batched(demag_plan* plan, int batch, int r, const float* lambda,
                                    const float* U, float* out_w, float* out_U, void* stream);

/* Tucker input (Eq. tucker_rep) -> Tucker output (Eq. kron_eval_tuck): the
 * core of component q is reused unchanged by the caller; term (k, q) has
 * weight c s omega_k and factors T_{k,q,p} V^(q,p).
 * r[3] >= 1 multilinear ranks; V: float blocks (q, p), each [r_p][n_p];
 * out_w: float [M][3]; out_V: three mode blocks, block p = [M][3][r_p][n_p]. */
demag_status demag_apply_tucker(demag_plan* plan, const int r[3], const float* V,
                                float* out_w, float* out_V, void* stream);
/* ---- Alg. 2 with compressed kernels (Sec. 4.2 Alg. 2; Alg. 1 HOOI; App. B) --
 * demag_compress_kernel compresses the CP convolution kernel of each
 * component (Eq. conv_pot: M terms of generator columns, weights c s omega_k)
 * to a Tucker tensor: QR of the generator matrices, HOSVD ranks by the rule
 * of Alg. 1 (discarded singular values of each unfolding <= tol/sqrt(3) of its
 * norm), the largest rank over the three components per mode, then HOOI
 * sweeps at those ranks; FP64 on the device, so ||K - K_tucker||_F <= tol ||K||_F.
 * It replaces any earlier compression of the plan and synchronizes `stream`.
 * tol in (0, 1).  Uniform grids whose FFT path exists only. */
demag_status demag_compress_kernel(demag_plan* plan, double tol, void* stream);
/* rho[p]: the Tucker ranks of the compressed kernels (shared by the components). */
demag_status demag_compressed_ranks(const demag_plan* plan, int rho[3]);
/* Device copies of the compressed kernels: gen (optional) double
 * [rhomax][3 q][3 p][2 nmax - 1] (row (i, q, p) = column i of U_p^(q), entries
 * d + n_p - 1 for |d| < n_p, zero past; rhomax = max rho), core (optional)
 * float [3 q][rho3][rho2][rho1].  Synchronous on `stream`. */
demag_status demag_copy_compressed(const demag_plan* plan, double* gen, float* core, void* stream);
/* Apply the compressed kernels to `batch` Tucker magnetizations (Alg. 2:
 * Lemma DFT_tucker and the Tucker Hadamard product of App. B Eq. t_had2, done
 * as circulant-FFT Toeplitz matvecs of the compressed generators).  Input as
 * demag_apply_tucker_batched plus the cores: core float [batch][3][r3][r2][r1],
 * V float blocks (q, p) [r_p][n_p] per item.  Output per item b and component q:
 * out_core float [batch][3][rho3 r3][rho2 r2][rho1 r1] = C^(q) (x) G^(q) with
 * index (i, l) = i r_p + l, and out_V: three mode blocks per item, block p =
 * [rho_p][3][r_p][n_p], row (i, q, l) = T(U_p^(q)[:, i]) V^(q,p)[:, l];
 * phi = sum_q [[out_core^(q); W^(q,1), W^(q,2), W^(q,3)]] with W^(q,p) column
 * (i, l) = row (i, q, l) of block p.  The core of a component has
 * prod_p rho_p r_p entries (the ranks multiply, App. B); with out_core NULL it
 * is left implicit as the Kronecker product of C^(q) (demag_copy_compressed)
 * and the input core, and core may then be NULL too.  FP32. */
demag_status demag_apply_tucker_compressed(demag_plan* plan, int batch, const int r[3], const float* core,
                                           const float* V, float* out_core, float* out_V, void* stream);

/* Alg. 2's approximate summation with tolerance tol: the output of
 * demag_apply_tucker_compressed for ONE item (core: its input cores G^(q),
 * float [3][r3][r2][r1]; V: its factor blocks, the out_V of that call) is
 * recompressed to one Tucker tensor phi_hat = [[C; U_1, U_2, U_3]] with
 * ||phi - phi_hat||_F <= tol ||phi||_F.  The range of each unfolding is sampled
 * with Khatri-Rao products of +-1 test vectors (16, 32, then 64 samples until
 * the projection error, computed exactly from the Tucker Gram matrices, is
 * below tol/2), the core projected, and an HOSVD of that core truncated with
 * the rank rule of Alg. 1 within the remaining error budget.  Outputs:
 * ranks_out[3]; core_out float [r3][r2][r1] (capacity 64^3); U_out float, per
 * mode p the rows [r_p][n_p] (orthonormal columns of U_p; capacity
 * 64 (n1 + n2 + n3)); err_out (optional, host) the relative error bound reached.
 * FP64 internally, synchronous.  DEMAG_EUNSUPPORTED when more than 64 ranks per
 * mode would be needed. */
demag_status demag_recompress_tucker(demag_plan* plan, const int r[3], const float* core, const float* V,
                                     double tol, int ranks_out[3], float* core_out, float* U_out,
                                     double* err_out, void* stream);

/* `batch` independent Tucker inputs in one launch per FFT length: item b of
 * V, out_w and out_V follows the single-item layout above at item strides
 * 3 sum_p r_p n_p, 3M and 3M sum_p r_p n_p floats.  batch >= 1. */
demag_status demag_apply_tucker_batched(demag_plan* plan, int batch, const int r[3], const float* V,
                                        float* out_w, float* out_V, void* stream);

/* Tensor train (App. C Eq. tt_3d_1, a 3D TT is the Tucker2 tensor
 * [[G2; G1, id, G3^T]], Eq. tt_3d_2) -> TT output: term (k, q) has weight
 * c s omega_k and cores T_{k,q,1} G1, T_{k,q,2} G2 (each mode-2 fibre),
 * T_{k,q,3} G3.  r[2] >= 1 TT ranks; G1: float [3][r1][n1],
 * G2: float [3][r1*r2][n2] (fibre index a1*r2 + a2), G3: float [3][r2][n3];
 * out_w: float [M][3]; oG1: float [M][3][r1][n1]; oG2: float [M][3][r1*r2][n2];
 * oG3: float [M][3][r2][n3]. */
demag_status demag_apply_tt(demag_plan* plan, const int r[2], const float* G1,
                            const float* G2, const float* G3, float* out_w, float* oG1,
                            float* oG2, float* oG3, void* stream);
/* `batch` independent TT inputs in one launch per FFT length: item b of each
 * array follows the single-item layout above, items one after another
 * (G1 item stride 3 r1 n1, G2 3 r1 r2 n2, G3 3 r2 n3, out_w 3M, oG_p M times
 * the input stride).  batch >= 1. */
demag_status demag_apply_tt_batched(demag_plan* plan, int batch, const int r[2], const float* G1,
                                    const float* G2, const float* G3, float* out_w, float* oG1,
                                    float* oG2, float* oG3, void* stream);

/* Tensor-train arithmetic of App. C, three components per call, layouts as
 * demag_apply_tt (G1 [3][r1][n1], G2 [3][r1 r2][n2] with row a1 r2 + a2,
 * G3 [3][r2][n3]); FP32, asynchronous, no allocation.
 * demag_tucker_to_tt: the Tucker magnetization (core float [3][r3][r2][r1],
 * V blocks (q, p) [r_p][n_p]) as trains of ranks (r1, r3), the second factor
 * multiplied into the core (the remark after Eq. tt_3d_2): G1 = V^(q,1),
 * G3 = V^(q,3), G2(a1, i2, a3) = sum_a2 G^(q)[a3][a2][a1] V^(q,2)[a2][i2].
 * demag_cp_to_tt: the CP magnetization (lambda float [3][r], U blocks (q, p)
 * [r][n_p]) as trains of ranks (r, r) with a diagonal middle core
 * G2(a1, i2, a2) = [a1 = a2] lambda_a1 U^(q,2)[a1][i2].
 * demag_tt_hadamard: C^(q) = A^(q) .* B^(q) element-wise as trains of ranks
 * (ra1 rb1, ra2 rb2) (the cores multiply as Kronecker products of their rank
 * indices): C1 row a rb1 + b, C2 row (a1 rb1 + b1)(ra2 rb2) + (a2 rb2 + b2),
 * C3 row a2 rb2 + b2. */
demag_status demag_tucker_to_tt(demag_plan* plan, const int r[3], const float* core, const float* V,
                                float* G1, float* G2, float* G3, void* stream);
demag_status demag_cp_to_tt(demag_plan* plan, int r, const float* lambda, const float* U, float* G1,
                            float* G2, float* G3, void* stream);
demag_status demag_tt_hadamard(demag_plan* plan, const int ra[2], const float* A1, const float* A2,
                               const float* A3, const int rb[2], const float* B1, const float* B2,
                               const float* B3, float* C1, float* C2, float* C3, void* stream);

/* TT rounding of the potential (App. C: the 3M output trains of
 * demag_apply_tt summed and rounded to one train, the recompression that
 * section cites) with tolerance tol: phi_hat = [G1, G2, G3] with
 * ||phi - phi_hat||_F <= tol ||phi||_F.  Inputs: the output of
 * demag_apply_tt for ONE item (r[2] its TT ranks; w float [M][3]; o1, o2, o3
 * its cores).  The range of the first unfolding is sampled with Khatri-Rao
 * products of +-1 test vectors (16, 32, then 64 samples until the projection
 * error, exact from the pairwise Gram matrices of the terms, is below tol/4),
 * the projected train's (1,2)-unfolding alike; the small train is truncated
 * as in TT-SVD (mode-1 Gram, QR of the middle core, Gram of the last core)
 * within the remaining budget, and the last core is the orthogonal projection
 * of phi on the first two.  Outputs: ranks_out[2]; G1_out float [r1][n1]
 * (orthonormal rows; capacity 64 n1); G2_out float [r1 r2][n2] (row
 * a1 r2 + a2; capacity 64^2 n2); G3_out float [r2][n3] (capacity 64 n3);
 * err_out (optional, host) = sqrt(1 - ||G3||^2 / ||phi||^2), the relative
 * error reached (exact up to a rounding floor near 1e-8).  FP64 internally,
 * synchronous.  DEMAG_EUNSUPPORTED when more than 64 samples per unfolding
 * would be needed; DEMAG_EINVAL for a zero potential. */
demag_status demag_round_tt(demag_plan* plan, const int r[2], const float* w, const float* o1,
                            const float* o2, const float* o3, double tol, int ranks_out[2],
                            float* G1_out, float* G2_out, float* G3_out, double* err_out, void* stream);

/* ---- stray field, energy and gradient (h_d = -grad phi, Sec. 1) ---------- */

/* Demag energy of a Tucker magnetization without forming a full tensor (Alg. 2
 * and the energy study after it): E = 1/2 h1 h2 h3 sum_q <m^(q), D_q phi>,
 * m^(q) = [[G^(q); V^(q,1), V^(q,2), V^(q,3)]], D_q the second-order difference
 * along axis q (the stencils of demag_stray_field) applied to the factors of
 * that axis, inner products of Tucker tensors through their factor Grams.
 * phi is the output of demag_apply_tucker for this input (out_w float [M][3],
 * out_V its three mode blocks).  r[3] in [1, 64]; core float [3][r3][r2][r1];
 * V float blocks (q, p) [r_p][n_p]; energy: one double on the device
 * (overwritten).  FP64 accumulation.  Uniform grids only. */
demag_status demag_energy_tucker(demag_plan* plan, const int r[3], const float* core, const float* V,
                                 const float* out_w, const float* out_V, double* energy, void* stream);

/* The same energy for a TT magnetization (Eq. tt_3d_1; G1 float [3][r1][n1],
 * G2 float [3][r1 r2][n2], G3 float [3][r2][n3]) from the output of
 * demag_apply_tt for it (out_w float [M][3], oG1, oG2, oG3): the inner
 * products of trains through the Grams of their first, middle and last cores.
 * r1, r2 in [1, 64] with r1 r2 <= 64; energy: one double on the device. */
demag_status demag_energy_tt(demag_plan* plan, const int r[2], const float* G1, const float* G2,
                             const float* G3, const float* out_w, const float* oG1, const float* oG2,
                             const float* oG3, double* energy, void* stream);

/* The same energy with phi given as one Tucker tensor [[phi_core; U_1, U_2, U_3]]
 * of ranks rho[3] in [1, 64] (the output of demag_recompress_tucker: phi_core
 * float [rho3][rho2][rho1], phi_U float rows [rho_p][n_p] per mode, modes one
 * after another). */
demag_status demag_energy_tucker_phi(demag_plan* plan, const int r[3], const float* core, const float* V,
                                     const int rho[3], const float* phi_core, const float* phi_U,
                                     double* energy, void* stream);

/* The energy of demag_energy_tucker with the Tucker application done here in
 * FP64 (the energy study after Alg. 2 on fine grids, where the FP32 factors of
 * demag_apply_tucker leave the energy about 5e-7 off): every factor
 * T_{k,q,p} V^(q,p) of Eq. kron_eval_tuck (E off the component's axis, F on
 * it) is summed directly from the plan's FP64 generators, O(n_p^2) per column,
 * then the Grams and the core contraction run in FP64.  core double
 * [3][r3][r2][r1]; V double blocks (q, p) [r_p][n_p]; r[3] in [1, 64]; energy:
 * one double on the device (overwritten).  Uniform grids with at most 8533
 * cells per axis (DEMAG_EUNSUPPORTED beyond); device memory for the factors is
 * taken and returned on the stream (cudaMallocAsync).  No counterpart in the
 * paper beyond its energy study. */
demag_status demag_energy_tucker_fp64(demag_plan* plan, const int r[3], const double* core, const double* V,
                                      double* energy, void* stream);

/* Second-order finite-difference stray field h_d = -D phi: central
 * differences inside, 3-point one-sided at the first and last cell of each
 * axis (two-point for n_p = 2, zero for n_p = 1).
 * phi: float [n3][n2][n1]; hd: float [3][n3][n2][n1] (overwritten). */
demag_status demag_stray_field(demag_plan* plan, const float* phi, float* hd, void* stream);

/* Demag energy E = -1/2 h1 h2 h3 sum_i m_i . h_d,i with h_d = -D P m, and
 * optionally its gradient dE/dm = 1/2 h1 h2 h3 (D P m + P^T D^T m).
 * m: float [3][n3][n2][n1]; energy: one double on the device (overwritten);
 * grad: float [3][n3][n2][n1] or NULL (energy only).  Uses `prec` for the
 * operator applications. */
demag_status demag_energy(demag_plan* plan, const float* m, double* energy, float* grad,
                          demag_precision prec, void* stream);

/* Stray field without finite differences: hd[p] = -d phi / d xi_p at the cell
 * centres, p = 1..3.  In the Kronecker form (Cor. 3) the collocation point
 * enters each 1D factor only through the limits of its cell integral, so the
 * derivative along axis p replaces the axis-p factors by dE = -2 tau_k^2 F and
 * dF[d] = b e^{-tau^2 b^2} - a e^{-tau^2 a^2} (a, b the cell limits; the
 * relations used for the micromagnetic stray field after Fig. 2), with 1/s for
 * the domain scaling.  Computed by the full-format chains of `prec` with the
 * derivative factors along one axis (the three directions share their first
 * stages: eight stage launches; with the fused schedule of demag_set_fused,
 * one fused launch and one mode-3 launch per direction, the derivative factors
 * along axis 1, 2 or 3).  m: float [3][n3][n2][n1]; hd: float
 * [3][n3][n2][n1] (overwritten).  Allocates the derivative factors on first
 * use of a precision. */
demag_status demag_stray_field_exact(demag_plan* plan, const float* m, float* hd, demag_precision prec,
                                     void* stream);

/* Read and clear the device-side status word of the plan (bounded waits that
 * gave up set DEMAG_ETIMEOUT there).  Synchronizes `stream`. */
demag_status demag_sync_status(demag_plan* plan, void* stream);

/* Limit of every bounded device-side wait of the plan's tensor-core kernels
 * (a pipeline barrier, a completion counter of an earlier tile), in seconds,
 * 0 <= seconds <= 60 (default 2).  A wait that runs out makes the kernel set
 * DEMAG_ETIMEOUT in the status word, let every copy and MMA it issued land,
 * release its tensor memory and return; demag_sync_status then reports it and
 * the plan stays usable.  For testing that failure path: limits this short
 * make normal runs fail.  Build-only; no counterpart in the paper. */
demag_status demag_set_wait_limit(demag_plan* plan, double seconds);

/* Schedule of the full-format forward application on tensor cores (BF16x3):
 * enable = 1 fuses the mode-1 and mode-2 products of Cor. 3
 * into one kernel on grids whose three axes are folded (longer than 16 cells)
 * with n1 and n2 at most 256: per slab i3 the mode-1 results are split
 * into hi / lo and used as the mode-2 operand in shared memory, never written
 * to the workspace; the mode-3 product reads the mode-2 fields in another
 * layout.  enable = 0 runs the three-stage chain (each mode product's fields
 * in the workspace).  The adjoint (demag_apply_adjoint, its first two
 * transposed mode products fused the same way) and the analytic stray field
 * (demag_stray_field_exact) take the same schedule.  Both give the same values
 * to rounding (the same
 * products, accumulated in another order); other grids and forms always run
 * the chain.  Without this call the plan takes the autotuner's choice
 * (demag_autotune, kind 9), else the fused schedule on grids of at least
 * 2^20 cells in the folded layout (about 100^3 and up) and the chain on
 * smaller ones.  Build-only; no counterpart in the paper. */
demag_status demag_set_fused(demag_plan* plan, int enable);

/* The forward schedule a plan's next full-format application in `prec`
 * takes: 1 the fused mode-1 / mode-2 kernel, 0 the three-stage chain, -1
 * when the plan has no tensor-core state for `prec` yet (no application or
 * demag_reserve_workspace in that form), `prec` is not a tensor-core form,
 * or plan is NULL.  A query; no error status is set.  Build-only; no
 * counterpart in the paper. */
int demag_forward_schedule(const demag_plan* plan, demag_precision prec);

/* ---- allocation-free full format (no counterpart in the paper) ---------- */

/* phi = sum_q P^(q) m^(q) exactly as demag_apply_full with DEMAG_FP32 (same
 * kernels, same order of operations), for callers that must not allocate
 * device memory: code running while a host framework's memory pool owns the
 * GPU (an allocation from a library would fail or fragment it), loops where
 * an allocation would implicitly synchronise the device, and hosts whose
 * plugin rules forbid allocation.  No plan is needed and nothing is
 * allocated: the nodes, generators, dense factors and intermediate fields
 * live in one fixed device array of 32 MiB inside the library, which every
 * GPU that loads the library keeps until the process exits.
 * desc: the grid, as for demag_build_factors; m: float [3][n3][n2][n1] and
 * phi: float [n3][n2][n1], device pointers owned by the caller.
 * Limits: the grid must fit the array: 8*(4M + 6M(2 nmax - 1)) + 8M sum_p
 * n_p^2 + 4(2M + 3) n1 n2 n3 bytes (each part rounded up to 256) <= 32 MiB
 * (for example 32^3 and 48^3 grids with R = 41 fit, 64^3 does not); larger
 * grids are rejected with DEMAG_EUNSUPPORTED and a message giving both sizes,
 * before anything is launched.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset, or anything else that destroys the device's primary
 * context, the module may be loaded again elsewhere and the kept address is
 * stale, so this call must not be used on that device again in the same
 * process.  Every call on a device uses the same array and leaves its
 * contents there; nothing in it has to start at zero.  Calls whose work can
 * overlap on the GPU (other streams, other host threads) race on the array:
 * serialise them.  Errors are reported through demag_last_error(NULL). */
demag_status demag_apply_full_noalloc(const demag_grid_desc* desc, const float* m, float* phi,
                                      void* stream);

/* ---- diagnostics (build-only; no counterpart in the paper) -------------- */

/* Number of kernels the library has launched for this plan so far. */
unsigned long long demag_launch_count(const demag_plan* plan);

/* Per-kernel-family timing.  demag_profile(plan, 1) clears the record and
 * brackets every later launch of the plan with CUDA events on its stream;
 * demag_profile(plan, 0) stops recording.  demag_profile_read sums the
 * recorded durations (milliseconds) and counts the launches of one family:
 * 0 = mode-product GEMM on CUDA cores, 1 = mode-product GEMM on tensor
 * cores, 2 = Toeplitz FFT, 3 = operand split / conversion, 4 = setup,
 * 5 = stray field / energy, 6 = small bookkeeping kernels (term weights),
 * 7 = passes of the 3D FFT convolution (demag_apply_full_fft).
 * Reading waits for the recorded events. */
demag_status demag_profile(demag_plan* plan, int enable);
demag_status demag_profile_read(demag_plan* plan, int family, double* total_ms, long long* launches);
/* The recorded launches one by one, in launch order: their number, and the
 * family and duration (ms) of record i.  Reading waits for its events. */
long long demag_profile_count(const demag_plan* plan);
demag_status demag_profile_launch(demag_plan* plan, long long i, int* family, double* ms);

/* ---- autotuning (build-only; no counterpart in the paper) --------------- */

/* demag_autotune(plan, 1) turns tuning on for this plan: from then on
 *  - the first Toeplitz-FFT launch of each shape (FFT length, number of column
 *    blocks, M) times every node-group size M, M/2, ..., 1 (one warm-up and
 *    three timed launches each, on the call's stream, which is synchronised)
 *    and keeps the fastest for later launches of that shape;
 *  - tensor-core state created afterwards (first DEMAG_TF32X3 / DEMAG_BF16X3
 *    use) times, per mode-product stage program, one knob after the other
 *    and keeps each at its fastest value: the output-column tile width
 *    {default, 128, 64} below the default, the operand stages {as many as
 *    fit, 4, 3, 2}, the tile order {every job of a row block in turn, every
 *    row block of a job in turn} and, where a 128-row block of the stage lies
 *    in one outer index, the store boxes {per epilogue warp, one 128-row box
 *    per chunk} (operands as they are, stage timed alone); then, where the
 *    grid has the fused BF16x3 forward schedule (demag_set_fused), that
 *    schedule's two launches against the three-stage chain.
 * No knob changes the arithmetic of an output element: tuned and untuned
 * results agree bit for bit.  The tuning launches write the call's own
 * outputs.  No tuning happens while the stream is being captured.
 * demag_autotune(plan, 0) stops tuning and keeps what was chosen. */
demag_status demag_autotune(demag_plan* plan, int enable);
/* Number of tuned shapes, and entry i of them: kind (0 FFT node group; tensor
 * cores, BF16x3 / TF32x3: 1 / 2 tile width, 3 / 4 operand stages (0 = as many
 * as fit), 5 / 6 tile order, 7 / 8 store boxes (1 = 128-row boxes); 9 the
 * BF16x3 forward schedule (1 fused, 0 chain)), key (FFT: log2 of the complex
 * FFT length, column blocks, M; tensor core: stage program 0..7 (6, 7: the
 * mode-3 stages of the fused forward and adjoint schedules), default value, 0;
 * schedule: 0, 1, 0, whatever the untuned choice), the chosen value, its time
 * per launch and the default value's time per launch in ms (for the schedule,
 * the untuned choice's time: fused from 2^20 folded cells, else the chain; 0
 * for an entry read from a cache). */
int demag_autotune_count(const demag_plan* plan);
demag_status demag_autotune_entry(const demag_plan* plan, int i, int* kind, int key[3], int* value, float* ms,
                                  float* ms_default);
/* Tuning cache: demag_autotune_save appends every entry of the plan to the
 * text file `path` (HOST path), one JSON object per line keyed by the current
 * GPU's UUID, the grid (n, R, uniform or not) and the entry's kind and key;
 * demag_autotune_load reads the lines of `path` that match the current GPU
 * and the plan's grid into the plan (a later line for the same entry wins;
 * *loaded, if not NULL, receives their count; a missing file loads nothing).
 * Load before the plan's first tensor-core use: its programs take the loaded
 * entries when they are built, and tuning then skips what is already chosen. */
demag_status demag_autotune_save(const demag_plan* plan, const char* path);
demag_status demag_autotune_load(demag_plan* plan, const char* path, int* loaded);

#ifdef __cplusplus
}
#endif

#endif /* DEMAG_H */
