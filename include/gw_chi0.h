/*
 * gw_chi0.h -- C ABI of the GB300 (sm_103a) independent-particle polarizability library.
 *
 * The library computes, on one GPU, the static/imaginary-frequency polarizability of
 * Eq. chi_mat of the SC'25 BerkeleyGW paper ("Overview of the Problem"):
 *
 *     chi_GG'(q, iw) = sum_{v,c} conj(M_vc(q,G)) Delta_vc(iw) M_vc(q,G')
 *
 * with the plane-wave matrix elements defined inline after Eq. ff-ch,
 *
 *     M_vc(G) = \int psi_v^*(r) e^{iG.r} psi_c(r) dr  (cell-normalised),
 *
 * evaluated in two stages: (a) the real-space pair product of the two bands on the
 * FFT grid, a forward FFT (sign +, scale 1/N_r) and a gather onto the caller's
 * G-sphere (the MTXEL step of the paper's Epsilon module); (b) the energy-weighted
 * Hermitian contraction over pairs (the CHI_SUM step, chunked over pairs like the
 * paper's NV-Block algorithm).  The energy factor, which the paper leaves open, is
 *
 *     Delta_vc(iw) = 2/(x - iw) + 2/(x + iw) = 4x/(x^2 + w^2),   x = E_v - E_c < 0,
 *
 * with w a non-negative imaginary-axis frequency in eV.  The paper's outer factor 2 is
 * folded into Delta; no volume or k-point normalisation is applied.
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved (re, im) pairs of doubles.
 *   - Pointers marked "device" are caller-owned CUDA device pointers valid for the
 *     duration of the call; pointers marked "host" are ordinary host memory.  The
 *     library keeps no caller pointer after a call returns.
 *   - All GPU work is enqueued on the stream given to gw_chi0_create; calls return
 *     after enqueueing (except where stated).  The caller synchronises the stream, or
 *     calls gw_chi0_sync, which also reports device-side errors.
 *   - No C++ exception crosses this boundary.  Each call returns a gw_status; on error
 *     a message is kept for gw_chi0_last_error and the handle stays usable.
 *   - Plane-wave vectors G are integer Miller triples (int32 [n][3]); a cubic cell with
 *     reciprocal vectors equal to the identity.
 *   - A handle serves one host thread at a time; calls on one handle from several threads
 *     must be serialised by the caller.  Separate handles share no state and may be used
 *     from separate threads (gw_chi0_contract_noalloc, which has no handle, excepted: see
 *     there).
 */
#ifndef GW_CHI0_H
#define GW_CHI0_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GW_API __attribute__((visibility("default")))
#else
#define GW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gw_chi0 gw_chi0; /* opaque, library-owned */

typedef enum {
    GW_OK = 0,
    GW_ERR_ARG = 1,         /* invalid argument (sizes, ranges, aliasing, energies) */
    GW_ERR_STATE = 2,       /* a required set_* call has not been made */
    GW_ERR_OOM = 3,         /* device allocation failed or the memory budget is too small */
    GW_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    GW_ERR_UNSUPPORTED = 5, /* request not supported by this build / device */
    GW_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up (reported by gw_chi0_sync) */
} gw_status;

/*
 * Contraction precision.  The value 2 (an Ozaki split on INT8 tensor cores, GW_PREC_OZAKI_INT8
 * in the method's statement) is deliberately absent: this GPU runs INT8 tensor instructions at
 * a small fraction of its BF16 rate (gw_chi0_probe measures both), so integer slices would
 * carry more work per useful bit on a slower pipe.  gw_chi0_create rejects it with GW_ERR_ARG.
 */
typedef enum {
    GW_PREC_FP64 = 0,      /* FP64 FFT + FP64 tensor-core (DMMA) contraction */
    GW_PREC_OZAKI_BF16 = 1 /* FP64 FFT + split-precision contraction on BF16 tensor cores */
} gw_prec;

typedef enum {
    GW_MTXEL_FP64 = 0,     /* stage (a) transforms in FP64 */
    GW_MTXEL_TWOFLOAT = 1  /* stage (a) pair transforms in two-float (FP32 pair, ~48-bit) arithmetic */
} gw_mtxel_prec;

typedef struct {
    int n[3];                /* FFT grid n0 x n1 x n2 (each a product of 2, 3, 5; 4 <= n <= 128) */
    int nq;                  /* number of q-point slots (>= 1) */
    int prec;                /* gw_prec */
    int nslices;             /* Ozaki slices for GW_PREC_OZAKI_BF16 (3..8); ignored for FP64 */
    int64_t pair_chunk;      /* pairs per M chunk; 0 = 8192 */
    size_t mem_budget_bytes; /* cap on library-owned device memory; 0 = no cap */
    int device;              /* CUDA device ordinal; must be current on the calling thread */
    int mtxel_prec;          /* gw_mtxel_prec */
    int single_stream;       /* 0: in split-precision streamed compute, the contraction of each chunk
                                runs on a second, high-priority stream beside the pair elements of
                                the next (tensor cores and FP32 pipes share the SMs); 1: every
                                kernel on the handle's stream, one after the other */
} gw_chi0_desc;

/*
 * Create a handle.  stream: a cudaStream_t (may be NULL for the legacy default stream).
 * Errors: GW_ERR_ARG (bad grid, nq < 1, prec/nslices/mtxel_prec out of range), GW_ERR_CUDA.
 */
GW_API gw_status gw_chi0_create(gw_chi0 **h, const gw_chi0_desc *d, void *cuda_stream);

/* Release every library-owned resource.  Safe on NULL. */
GW_API void gw_chi0_destroy(gw_chi0 *h);

/* Message of the last failed call on this handle ("" if none).  Owned by the handle. */
GW_API const char *gw_chi0_last_error(const gw_chi0 *h);

/* Make subsequent calls enqueue on another stream (e.g. the caller's current stream). */
GW_API gw_status gw_chi0_set_stream(gw_chi0 *h, void *cuda_stream);

/*
 * Band setup (step a1): psi_n(r) = sum_K c_n(K) e^{+iK.r} on the n0 x n1 x n2 grid (no
 * 1/N factor), kept in library-owned device memory [nb][n0][n1][n2] complex128.
 *   iq      q slot for valence bands (0 <= iq < nq); conduction bands (kind = 1) are
 *           shared by every slot and iq is ignored.
 *   kind    0 = valence (bands at k+q), 1 = conduction (bands at k).
 *   gvec    device int32 [ngpsi][3]  plane waves of the coefficient rows.
 *   coeff   device complex128 [nb][ngpsi].
 *   energy  device float64 [nb], eV.
 * Validation (GW_ERR_ARG): nb, ngpsi >= 1; |G| components inside (-n/2, n/2); every
 * valence energy below every conduction energy once both sets are present.  Reads gvec
 * and energy back to the host (synchronous on the stream).
 */
GW_API gw_status gw_chi0_set_bands(gw_chi0 *h, int iq, int kind, int nb, int ngpsi, const int32_t *gvec,
                            const double *coeff, const double *energy);

/*
 * Dielectric G-sphere of slot iq (the G, G' index set of chi).  gvec: device int32 [ng][3].
 * Errors (GW_ERR_ARG): ng < 1; the set is not alias-free for the stored bands, i.e.
 * 2 max|K| + max|G| >= n on some axis.
 */
GW_API gw_status gw_chi0_set_gsphere(gw_chi0 *h, int iq, int ng, const int32_t *gvec);

/*
 * Forward chi0 for nq slots and nw imaginary frequencies (steps a1-a7 after setup).  With
 * two-float stage (a) on the 48^3 grid the last axis of the pair transform runs on the BF16
 * tensor cores (the route of gw_chi0_pair_elements_block); elsewhere stage (a) is the pruned
 * FFT pair kernel.
 *   iq     host int [nq]      slots to compute.
 *   omega  host double [nw]   imaginary-axis frequencies w >= 0 (eV).
 *   chi    device complex128, packed by slot: for slot i, nw blocks of ng_i x ng_i
 *          (row G, column G'), slot blocks consecutive in the order of iq.  Written in
 *          full (exactly Hermitian, zero imaginary diagonal); not accumulated into.
 *   diag   device float64 or NULL: same packing, nw x ng_i values chi_GG computed by an
 *          independent column reduction of Delta |M|^2 (a trace check).
 * Errors: GW_ERR_STATE (bands or sphere missing), GW_ERR_ARG, GW_ERR_OOM, GW_ERR_CUDA.
 */
GW_API gw_status gw_chi0_compute(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, double *chi,
                          double *diag);

/*
 * Batched forward chi0 (step a8): the same result and output packing as gw_chi0_compute,
 * for many slots and frequencies at once.  Every requested slot's matrix elements are
 * produced once and kept resident (library memory: sum over slots of P_q x N_G(q) x 16
 * bytes, plus the split slices of one frequency in GW_PREC_OZAKI_BF16 mode); the
 * contraction of all (q, w) blocks then runs as one persistent launch (FP64) or one
 * persistent launch per frequency covering every slot (split precision), ordered largest
 * block first.  The whole sequence is captured once per call signature (slots, sphere
 * sizes, frequencies, output pointers) into a CUDA graph and replayed on later calls.
 * On the first call of a problem shape an autotuner times the contraction's launch-shape
 * candidates (FP64 tile edge 32/64 and wave count; split-precision tile width 128/240/256
 * columns) and keeps the fastest for the handle (see gw_chi0_tuning).  The first call
 * synchronises the stream; replays are asynchronous.  Slots must be distinct.
 * Errors: as gw_chi0_compute; GW_ERR_OOM when the resident buffers do not fit.
 */
GW_API gw_status gw_chi0_compute_batch(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, double *chi,
                                       double *diag);

/*
 * Launch shapes in use (chosen by the autotuner of gw_chi0_compute_batch, or defaults):
 * FP64 tile edge (complex), FP64 waves, split-precision tile width (real columns; 256 before
 * tuning, when each contraction instead takes 240 or 256 columns by which fills the SMs' waves
 * better).  The environment variable GW_CHI0_SPLIT_TILE=128, 240 or 256, read at every
 * contraction, forces the split-precision tile width; the results do not depend on it.
 * Returns the number of problem shapes tuned so far.  Any pointer may be NULL.
 */
GW_API int gw_chi0_tuning(const gw_chi0 *h, int *tile_f64, int *waves_f64, int *tile_split);

/*
 * Stage (a) alone (steps a2-a4): M[p - pair_begin][g] for pairs p = v*nc + c in
 * [pair_begin, pair_begin + pair_count) of slot iq.  M: device complex128 [pair_count][ng].
 */
GW_API gw_status gw_chi0_pair_elements(gw_chi0 *h, int iq, int64_t pair_begin, int64_t pair_count, double *M);

/*
 * Stage (a) alone for all valence bands of slot iq and the conduction bands c0 .. c0 + cb - 1,
 * on the route gw_chi0_compute takes for two-float stage (a) on the 48^3 grid: the last-axis
 * transform of the pair products as a split product on the BF16 tensor cores (the grid line's
 * valence points against the conduction points times the kept twiddles, six BF16 slices each,
 * FP32 group sums combined in two-float arithmetic), the middle and first axes as in the FFT
 * pair kernel.  Rows in that route's order: M[(c - c0) nv + v][g], device complex128
 * [cb nv][ng].  GW_ERR_UNSUPPORTED when the slot does not take the route (another grid, FP64
 * stage (a), resident pair elements kept); GW_ERR_ARG for a block outside [0, nc).  Uses the
 * handle's work buffers (the last-axis output of cb nv pairs, 16 * 48^2 * K2 bytes per pair).
 */
GW_API gw_status gw_chi0_pair_elements_block(gw_chi0 *h, int iq, int c0, int cb, double *M);

/*
 * Stage (b) alone (steps a5-a7) on caller-given matrix elements, using the handle's
 * precision mode:  chi[w][G][G'] = sum_p conj(M[p][G]) Delta_p(w) M[p][G'],
 * p = v*nc + c, Delta from ev [nv] and ec [nc] (device float64, eV).
 *   M     device complex128 [nv*nc][ng]
 *   omega host double [nw]
 *   chi   device complex128 [nw][ng][ng], written in full.
 * Needs no set_* call.
 */
GW_API gw_status gw_chi0_contract(gw_chi0 *h, int nv, int nc, const double *ev, const double *ec, int ng,
                           const double *M, int nw, const double *omega, double *chi);

/*
 * Static subspace approximation (Eq. chi_mat_sub and the paragraph around it): chi(w = 0) is
 * diagonalised and its neig most significant eigenvectors (chi(0) is negative semidefinite:
 * the most negative eigenvalues) form the N_G x N_Eig projection matrix C_s.
 *   chi0   device complex128 [ng][ng], Hermitian (read only).
 *   basis  device complex128 [ng][neig]: C_s, column B the eigenvector of eigenvalue B
 *          (ascending, most significant first); each column's phase is arbitrary.
 *   evals  device float64 [neig] or NULL: the eigenvalues.
 * One dense eigendecomposition (cuSOLVER zheevdx, only the wanted vectors, loaded on first
 * use; GW_ERR_UNSUPPORTED when it is not installed).  Synchronises the handle's stream.
 * GW_ERR_ARG unless 1 <= neig <= ng.
 */
GW_API gw_status gw_chi0_subspace_basis(gw_chi0 *h, int ng, const double *chi0, int neig, double *basis,
                                        double *evals);

/*
 * chi_BB'(i w) = sum_vc conj(M^B_vc) Delta_vc(i w) M^B'_vc with M^B_vc = sum_G M_vc(G) C_s[G][B]
 * (Eq. chi_mat_sub), for slot iq: per pair chunk, stage (a), the projection onto C_s (split
 * precision on the BF16 tensor cores, or FP64 DMMA, following the handle's mode), then stage
 * (b) on the neig columns.  Equals C_s^H chi(i w) C_s.
 *   basis    device complex128 [ng][neig] (e.g. from gw_chi0_subspace_basis).
 *   omega    host double [nw], imaginary-axis magnitudes (eV).
 *   chi_sub  device complex128 [nw][neig][neig], written in full, Hermitian.
 * Errors as gw_chi0_compute; GW_ERR_ARG unless 1 <= neig <= ng of the slot's sphere.
 */
GW_API gw_status gw_chi0_compute_subspace(gw_chi0 *h, int iq, int neig, const double *basis, int nw,
                                          const double *omega, double *chi_sub);

/*
 * Forward derivative (JVP) of chi0(iq, i w) along a perturbation of the stored bands: the
 * first-order change the GWPT working equation (Eq. gwpt) builds from d psi_n,
 *     dchi = sum_p [conj(dM_p) Delta_p M_p + conj(M_p) Delta_p dM_p + conj(M_p) dDelta_p M_p],
 *     dM_vc = M(d psi_v, psi_c) + M(psi_v, d psi_c),  dDelta = dDelta/dx (dE_v - dE_c),
 * computed per chunk with the pair kernel on the tangent grids and the stage-(b) kernels
 * (the cross term as [chi(M + dM) - chi(M - dM)] / 2).
 *   dcoeff_v device complex128 [nv][ngpsi_v], dcoeff_c [nc][ngpsi_c]: the tangent coefficients,
 *            on the plane waves of the stored band sets (no re-orthonormalisation).
 *   dE_v     device float64 [nv]; dE_c [nc]: the tangent energies.
 *   omega    host double [nw] (imaginary-axis magnitudes, eV), nw <= 32.
 *   dchi     device complex128 [nw][ng][ng], written in full, Hermitian.
 * Work buffers for the tangent grids are held for the call only.  Errors as gw_chi0_compute.
 */
GW_API gw_status gw_chi0_jvp(gw_chi0 *h, int iq, int nw, const double *omega, const double *dcoeff_v,
                             const double *dcoeff_c, const double *dE_v, const double *dE_c, double *dchi);

/*
 * chi0 on the real frequency axis with broadening eta (Eq. chi_mat with Delta continued from
 * the imaginary axis, i w -> w + i eta):
 *     Delta_vc(w) = 2/(x - w - i eta) + 2/(x + w + i eta),  x = E_v - E_c,
 *     chi(w) = sum_vc conj(M_vc(G)) Delta_vc(w) M_vc(G') = chi_R + i chi_I,
 * with chi_R, chi_I the Hermitian contractions with Re Delta and Im Delta (Im Delta <= 0 for
 * w >= 0; Re Delta changes sign near the resonances and is split into its two signs).
 *   omega  host double [nw], real frequencies >= 0 (eV), nw <= 21.
 *   eta    broadening > 0 (eV).
 *   chi    device complex128 [nw][ng][ng], written in full (not Hermitian).
 * Errors as gw_chi0_compute.
 */
GW_API gw_status gw_chi0_compute_real(gw_chi0 *h, int iq, int nw, const double *omega, double eta, double *chi);

/*
 * Inverse dielectric matrix, Eq. epsilon_mat: epsinv(w) = [I - v chi(w)]^-1 with v the diagonal
 * Coulomb matrix, for nw Hermitian, negative semidefinite chi blocks.
 *   chi     device complex128 [nw][ng][ng] (e.g. from gw_chi0_compute).
 *   vcoul   device float64 [ng]: v_G > 0 (the caller's Coulomb form, e.g. 4 pi / |q + G|^2).
 *   epsinv  device complex128 [nw][ng][ng], written in full.
 * Method: the Hermitian A = I - s chi s (s = sqrt(v), eigenvalues >= 1) is inverted by the
 * Newton-Schulz iteration X <- 2X - X A X from X0 = 2/(1 + b) I, b a Gershgorin bound,
 * with the step count that brings the error below 1e-17 from (b-1)/(b+1); the products run
 * in the handle's precision mode.  Then epsinv = s X s^-1.  Synchronises once per block.
 * In split precision the result's error is the rounding of the last steps' products (earlier
 * errors are squared away), so the last two steps use 8 slices whatever the handle's count
 * (N_G = 2000, chi of the 48^3 workload: 3e-11 against a dense FP64 inverse; 2e-9 with 7).
 * GW_ERR_ARG for v <= 0 or when I - v chi is not positive.
 */
GW_API gw_status gw_chi0_epsilon_inverse(gw_chi0 *h, int ng, int nw, const double *chi, const double *vcoul,
                                         double *epsinv);

/*
 * Full-matrix (off-diagonal) self-energy of the plasmon-pole model on an energy grid -- the
 * Sigma-module kernel of the section on the off-diagonal GPP kernel, whose work is the two
 * products per (n, E) counted by Eq. flop_count_fullmat:
 *   sigma[e][l][m] = sum_n sum_{G,G'} conj(M[n][l][G]) P^n_GG'(E[e]) M[n][m][G'],
 *   P^n_GG'(E) = v[G'] Omega2[G][G'] / (2 wt[G][G'] (E - En[n] - s_n wt[G][G'])),
 * s_n = -1 for an occupied band (n < nocc), +1 otherwise: the correlation part of the
 * Hybertsen-Louie plasmon-pole model the paper cites for the frequency dependence (its working
 * equation is in a figure).  P^n(E) is formed per (n, E) (the prep. step) and never leaves the
 * device; in split-precision mode it goes straight into BF16 column slices.
 *   nb, nocc  summed bands n and how many of them (the first nocc) are occupied; 0 <= nocc <= nb.
 *   nsig, ng  self-energy bands l, m and plane waves G (the dielectric sphere).
 *   M       device complex128 [nb][nsig][ng], M[n][l][G] (e.g. from gw_chi0_pair_elements).
 *   En      host double [nb], band energies (eV).
 *   omega2  device complex128 [ng][ng], Omega^2_GG' (eV^2).
 *   wtilde  device complex128 [ng][ng], mode energies (eV); keep E - En[n] -+ wt away from 0
 *           (a damping Im wt != 0 does).
 *   vcoul   device float64 [ng], the Coulomb diagonal v_G.
 *   ne, E   host double [ne], the energy grid (eV); ne = 0 is a no-op.
 *   sigma   device complex128 [ne][nsig][nsig], written in full (zero when nb = 0).
 * Work buffers, held by the handle until destroy: FP64 mode two [ng][ng] complex128 matrices;
 * split mode the pole parameters transposed in two-float form (32 ng^2 bytes), the BF16 slices
 * of P^T for a batch of energies (28 ng^2 bytes each at 7 slices, at most 32 GiB or a quarter of
 * mem_budget_bytes when set) and X^T for 16 energies (16 nsig ng complex128 plus its slices).
 * GW_ERR_ARG for sizes out of range, null or misaligned (16 bytes) complex pointers, non-finite
 * energies; other errors as gw_chi0_compute.
 */
GW_API gw_status gw_chi0_sigma_gpp(gw_chi0 *h, int nb, int nocc, int nsig, int ng, const double *M, const double *En,
                                   const double *omega2, const double *wtilde, const double *vcoul, int ne,
                                   const double *E, double *sigma);

/*
 * Adjoint of L = Re Tr(W chi0(iq, w)) (GWPT-style sensitivity, Eq. gwpt motivates it).
 * Matrix elements are recomputed chunk by chunk; Y = M W_h runs as a split product on the
 * BF16 tensor cores in split-precision mode, on DMMA otherwise.
 *   W        device complex128 [ng][ng], any complex matrix (read only).  chi0 is Hermitian, so
 *            L depends on W only through its Hermitian part W_h = (W + W^H)/2, which the call
 *            forms itself: an upstream gradient dL/dchi in torch's convention (dL/dRe + i dL/dIm,
 *            equal to W^H for this L) can be passed as it is.
 *   L        host double* or NULL: the value of L (synchronous when non-NULL).
 *   dE_v     device float64 [nv]; dE_c device float64 [nc]: dL/dE.
 *   dcoeff_v device complex128 [nv][ngpsi_v]; dcoeff_c [nc][ngpsi_c]:
 *            dL/dRe c + i dL/dIm c for every coefficient of the stored band sets.
 * Outputs are written in full.  Errors as gw_chi0_compute.
 */
GW_API gw_status gw_chi0_adjoint(gw_chi0 *h, int iq, double omega, const double *W, double *L, double *dE_v,
                          double *dE_c, double *dcoeff_v, double *dcoeff_c);

/*
 * Keep pair elements resident (enable = 1): gw_chi0_compute then writes the M of each slot it
 * computes into a library-owned buffer (P x N_G complex128, 4.2 GB on the 48^3 workload) instead
 * of one chunk buffer, and gw_chi0_compute_subspace / gw_chi0_compute_real / gw_chi0_jvp on the
 * last slot computed reuse it (stage (a) skipped; the JVP still forms its two tangent products).  The buffer is taken only when it fits the handle's memory
 * budget (when one is set) and half the free device memory; otherwise compute runs as without.
 * gw_chi0_set_bands / gw_chi0_set_gsphere of that slot (or of the conduction set) drop the
 * elements.  enable = 0 (the default) frees the buffer.  GW_ERR_ARG for other values.
 */
GW_API gw_status gw_chi0_keep_pair_elements(gw_chi0 *h, int enable);

/*
 * How many streams a single-frequency gw_chi0_compute uses for slot iq as it stands (bands and
 * sphere set): 2 when each chunk's split contraction runs on a second stream beside the next
 * chunk's pair elements (split precision, two-float stage (a) by the FFT pair kernel, and room for
 * two pair-kernel blocks beside a contraction block on an SM), else 1 (always 1 on the
 * tensor-core route of stage (a), see gw_chi0_pair_elements_block).  Calls with several frequencies always
 * run on one stream.  Negative (a gw_status, negated) on a bad handle or slot.
 */
GW_API int gw_chi0_streams(gw_chi0 *h, int iq);

/*
 * Synchronise the handle's stream and report device-side status: GW_ERR_TIMEOUT if a
 * bounded wait inside a kernel gave up since the last gw_chi0_sync, GW_ERR_CUDA on a
 * CUDA error, else GW_OK.  Clears the device status word.
 */
GW_API gw_status gw_chi0_sync(gw_chi0 *h);

/*
 * Failure-detection check: enqueue one device wait, bounded by `iterations` tries, on an
 * mbarrier that nothing arrives at -- the same bounded wait the contraction kernels use on
 * their TMA and MMA barriers.  When the bound runs out the kernel records a timeout in the
 * handle's status word and returns; the next gw_chi0_sync reports GW_ERR_TIMEOUT and the
 * handle (and CUDA context) stay usable.  Nothing faults, traps or hangs.
 */
GW_API gw_status gw_chi0_check_watchdog(gw_chi0 *h, long long iterations);

/*
 * Per-kernel timing.  When enabled, every library kernel launch is bracketed by CUDA
 * events on the handle's stream.  gw_chi0_timing fills, for up to n kernel classes,
 * names (host char[n][32]), total milliseconds and launch counts since the last reset
 * (synchronises the stream).  Returns the number of classes.
 */
GW_API gw_status gw_chi0_set_timing(gw_chi0 *h, int enable);
GW_API int gw_chi0_timing(gw_chi0 *h, int n, char (*names)[32], double *ms, int64_t *launches, int reset);

/* Library-owned device bytes currently held by the handle. */
GW_API size_t gw_chi0_device_bytes(const gw_chi0 *h);

/*
 * Peak-rate probes (measurement helper; no counterpart in the paper).  Enqueues one launch on
 * the given stream (a cudaStream_t, NULL = legacy default) that fills every SM of the current
 * device with independent chains of one instruction kind, `iters` instructions per chain, and
 * returns in *ops the arithmetic operations it performs (an FMA counts 2, a tensor instruction
 * 2 m n k).  The caller times the launch (CUDA events) and divides.  These rates are the
 * denominators of the roofline fractions of kernels bound by those pipes: FP32 FMA (scalar and
 * packed two-lane), FP64 FMA, FP64 tensor (DMMA), and the warp-level BF16 / INT8 tensor
 * instructions.  sink: device float32 [256], written only if a chain takes an impossible value
 * (it keeps the chains from being optimised away).  GW_ERR_ARG for an unknown kind, iters < 1 or
 * null pointers; GW_ERR_CUDA if the launch fails.
 */
typedef enum {
    GW_PROBE_FFMA = 0,           /* fma.rn.f32 */
    GW_PROBE_FFMA2 = 1,          /* fma.rn.f32x2 (two lanes per instruction) */
    GW_PROBE_FADD2 = 2,          /* add.rn.f32x2 */
    GW_PROBE_DFMA = 3,           /* fma.rn.f64 */
    GW_PROBE_DMMA_M8N8K4 = 4,    /* mma.sync m8n8k4 f64 */
    GW_PROBE_DMMA_M16N8K16 = 5,  /* mma.sync m16n8k16 f64 */
    GW_PROBE_BF16_MMA_SYNC = 6,  /* mma.sync m16n8k16 bf16 -> f32 (warp-level, not tcgen05) */
    GW_PROBE_INT8_MMA_SYNC = 7,  /* mma.sync m16n8k32 s8 -> s32 (warp-level, not tcgen05) */
    GW_PROBE_TCGEN05_N64 = 8,    /* tcgen05.mma kind::f16 BF16 M=128 N=64 K=16 from shared memory */
    GW_PROBE_TCGEN05_N128 = 9,   /* the same, N = 128 */
    GW_PROBE_TCGEN05_N256 = 10   /* the same, N = 256 */
} gw_probe_kind;
GW_API gw_status gw_chi0_probe(int kind, long long iters, void *cuda_stream, float *sink, double *ops);

/*
 * gw_chi0_contract_noalloc -- stage (b) in FP64 without any device allocation.
 *
 * The paper has no counterpart to this call.  It serves callers that cannot call
 * cudaMalloc: plugins whose host framework owns every device allocation through its own
 * pool (an allocation behind the pool's back fragments it, or fails once the pool holds the
 * free memory), and services that forbid allocator calls on their hot path (cudaMalloc and
 * cudaFree can synchronise the device and take unbounded time).  It computes what
 * gw_chi0_contract computes in GW_PREC_FP64 mode (same kernels, same arguments and layouts,
 * chi written in full), without a handle, on the given stream (a cudaStream_t; NULL =
 * legacy default stream), for the current device.
 *
 * Its only scratch -- the energy factors Delta of every pair and frequency, the kernel's
 * job table and a status word -- lives in one fixed device array compiled into the library
 * (4 MiB + 16.25 KiB; every GPU that loads the library holds it until the process exits).
 *   - Limit: nw * nv * nc <= 524288; larger requests return GW_ERR_ARG and do nothing.
 *   - The first call on a device looks up that array's device address (once per device,
 *     with the device current); make that first call before any stream capture.
 *   - The job table goes up with one cudaMemcpyAsync from host memory of the calling
 *     thread (staged by the driver; the call returns after the host side of the copy).
 *   - Every call shares the array and finds the previous call's contents there: calls that
 *     overlap on the GPU (other streams, other host threads) race on it and must be
 *     serialised by the caller.  The status word is cleared at the start of each call.
 *   - A bounded device-side wait that gives up cannot be reported through the return
 *     value (the call returns before the kernels run); the call then writes NaN on the
 *     diagonal of every chi block, so a partial result cannot pass as a valid one.
 * Calls no cudaMalloc, cudaFree or allocating library routine.  Returns GW_OK,
 * GW_ERR_ARG (null pointers, sizes out of range, M not 16-byte aligned, bad omega),
 * GW_ERR_CUDA, or GW_ERR_UNSUPPORTED (device ordinal >= 64).
 */
GW_API gw_status gw_chi0_contract_noalloc(int nv, int nc, const double *ev, const double *ec, int ng,
                                          const double *M, int nw, const double *omega, double *chi,
                                          void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GW_CHI0_H */
