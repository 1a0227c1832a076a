// Internal launch interface between the host API and the kernel translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include "common.cuh"

namespace gw {

constexpr int kMaxOmega = 64;
struct OmegaList {
    int nw;
    double w[kMaxOmega];
};

// ---- stage (a): band setup and pair elements (mtxel.cu)
cudaError_t launch_scatter(const double2 *coeff, const int32_t *gofs, int nb, int ngpsi, int64_t nr, double2 *psi,
                           cudaStream_t st);
cudaError_t launch_band_fft(double2 *psi, int nb, const int n[3], const FftAxis ax[3], cudaStream_t st);

struct PairPlan {
    int n[3];
    FftAxis ax[3];
    int K2;              // number of needed frequencies along the last axis
    const int *kz;       // device [K2]   needed last-axis frequencies (0..n2-1)
    int ng;
    const int32_t *gpack; // device [ng]   k0 | k1 << 8 | k2index << 16
    int K12;              // number of (k1, k2) cells that hold sphere points
    const int32_t *cell;  // device [K12]  k2index << 8 | k1, ordered by (k2index, k1)
    const int *cstart;    // device [K12 + 1] points of cell d: cpts[cstart[d] .. cstart[d + 1])
    const int2 *cpts;     // device [ng]   (point index, k0 | cell << 8), grouped by cell
    // scratch of the two-float grid-specialised kernel (pair_tf_scratch): nslots slots of
    // n0 * K12 two-float values, one flag per slot
    float4 *scr;
    int *slot_flags;
    int nslots;
    int *status;          // device status word (kStatusNoSlot)
};
// Scratch the two-float pair kernel needs for a plan: *nslots slots of *slot_elems float4
// (0 slots: the plan runs on the runtime-shape kernel, which needs none).
cudaError_t pair_tf_scratch(const PairPlan &pp, int *nslots, size_t *slot_elems);
// Shared memory per block of the grid-specialised two-float pair kernel for this plan (0 when it
// does not take the plan).
size_t pair_tf_ct_smem_bytes(const PairPlan &pp);
// M[p - p0][g] for p in [p0, p0 + count); pair p = v * nc + c.
cudaError_t launch_pair(const double2 *psiv, const double2 *psic, int nc, int64_t p0, int64_t count,
                        const PairPlan &pp, double2 *M, cudaStream_t st);
int pair_max_ng();
// the same in two-float arithmetic; psiv/psic hold two-float grids (launch_band_setup_tf)
cudaError_t launch_pair_tf(const void *psiv, const void *psic, int nc, int64_t p0, int64_t count,
                           const PairPlan &pp, double2 *M, cudaStream_t st);
// band setup in two-float arithmetic: scatter (with hi/lo split) + 3D FFT, psi in two-float form
// maxabs: largest |G_a| of the plane waves (input pruning of the grid-specialised transforms)
cudaError_t launch_band_setup_tf(const double2 *coeff, const int32_t *gofs, int nb, int ngpsi, void *psi,
                                 const int n[3], const FftAxis ax[3], const int maxabs[3], cudaStream_t st);


// ---- stage (a) last-axis transform on the tensor cores (zdft.cu) and the rest of the pair
// transform from its output (pair_tf_ct.cuh)
constexpr int kZdSlices = 6; // BF16 slices per operand (balanced base-256 digits)
// valence slices A[kZdSlices][n^2 lines][nv][2n] (BF16) of two-float band grids psiv [nv][n^3]
cudaError_t launch_zd_aslices(const void *psiv, int nv, int n, uint16_t *A, cudaStream_t st);
bool zd_supported(int n, int K2, int nv);
int zd_conduction_per_tile(int K2);
size_t zd_smem_bytes(int n, int K2);
// F[l][cl nv + v][q] (two-float) = sum_i2 conj(psi_v[l][i2]) W^{kz[q] i2} psi_c[l][i2] for the
// conduction bands c = c0 + cl, cl < cb; tmA maps the valence slices (box {32, 128, 1, 6},
// 64-byte swizzle)
// tmC maps the conduction grids as FP32 [nc][n^2 lines][4n], box {4n, 1, zd_conduction_per_tile(K2)}
cudaError_t launch_zd_gemm(const CUtensorMap &tmA, const CUtensorMap &tmC, const void *psic, const int *kz,
                           const float4 *twf, int n, int nv, int c0, int cb, int K2, float4 *F, int *status,
                           cudaStream_t st);
// M[r][g] of the chunk's R pairs from F (middle and first axis of the pair transform)
// (tmF: F as [N^2 lines][R K2] two-float entries, FP32 elements, box {4 K2, 2 N}; tmS: the plan's
// scratch slots as [nslots N rows][K12] two-float entries, box {8 K2, N}; no swizzle)
cudaError_t launch_pair_tf_from_f(const CUtensorMap &tmF, const CUtensorMap &tmS, int64_t R, const PairPlan &pp,
                                  double2 *M, cudaStream_t st);
// delta[w][cl nv + v] = 4x/(x^2 + w^2), x = ev[v] - ec[c0 + cl], the row order of the chunks above
cudaError_t launch_delta_block(const double *ev, const double *ec, int nv, int c0, int cb, const OmegaList &om,
                               double *delta, cudaStream_t st);

// ---- energy factor, diagonal, symmetrisation (reduce.cu)
// delta[w][p - p0] = 4x/(x^2 + w^2), x = ev[v] - ec[c]
cudaError_t launch_delta(const double *ev, const double *ec, int nc, int64_t p0, int64_t count, const OmegaList &om,
                         double *delta, cudaStream_t st);
// real axis with broadening: delta[3w + k][p - p0], k = 0: min(Re D, 0), 1: -max(Re D, 0), 2: Im D
cudaError_t launch_delta_real(const double *ev, const double *ec, int nc, int64_t p0, int64_t count,
                              const OmegaList &om, double eta, double *delta, cudaStream_t st);
// out[w] = (T[3w] - T[3w+1]) + i T[3w+2]
cudaError_t launch_combine_real(const double2 *T, int64_t nn, int nw, double2 *out, cudaStream_t st);
// forward derivative of Delta along (dE_v, dE_c), split: out[2w] = min(dD, 0), out[2w+1] = -max(dD, 0)
cudaError_t launch_delta_jvp(const double *ev, const double *ec, const double *dev, const double *dec, int nc,
                             int64_t p0, int64_t count, const OmegaList &om, double *out, cudaStream_t st);
// d = X1 + X2; X1 = M + d; X2 = M - d
cudaError_t launch_jvp_mix(const double2 *M, double2 *X1, double2 *X2, int64_t n, cudaStream_t st);
// out[w] = (Tp[w] - Tm[w]) / 2 + Tw[2w] - Tw[2w+1]
cudaError_t launch_combine_jvp(const double2 *Tp, const double2 *Tm, const double2 *Tw, int64_t nn, int nw,
                               double2 *out, cudaStream_t st);
// diag[w][g] += sum_p delta[w][p] |M[p][g]|^2
cudaError_t launch_diag(const double2 *M, int64_t P, int ng, const double *delta, int64_t dstride, int nw,
                        double *diag, int64_t diag_wstride, cudaStream_t st);
// ---- dielectric matrix inverse (epsilon.cu)
cudaError_t launch_eps_sqrt(const double *v, int ng, double *sv, cudaStream_t st);
// A = I - s chi s and bmax = Gershgorin bound of A (bits of a double)
cudaError_t launch_eps_sym(const double2 *chi, const double *sv, int ng, double2 *A, unsigned long long *bmax,
                           cudaStream_t st);
cudaError_t launch_eps_init(double2 *X, int ng, const unsigned long long *bmax, cudaStream_t st);
cudaError_t launch_eps_step(double2 *X, const double2 *P, int64_t n, cudaStream_t st);
cudaError_t launch_eps_unsym(const double2 *X, const double *sv, int ng, double2 *out, cudaStream_t st);

// out[g][b] = conj(V[b n + g]) (column-major n x neig -> row-major [n][neig], conjugated)
cudaError_t launch_conj_transpose(const double2 *V, int n, int neig, double2 *out, cudaStream_t st);
// a bounded wait that is never satisfied: sets kStatusTimeout in *status after iters tries
cudaError_t launch_watchdog(long long iters, int *status, cudaStream_t st);
// out = (W + W^H) / 2 for a row-major n x n complex matrix (out must not alias W)
cudaError_t launch_herm_part(const double2 *W, int n, double2 *out, cudaStream_t st);
// lower triangle <- conj(upper), Im diag <- 0, for nw consecutive ng x ng blocks
cudaError_t launch_symmetrize(double2 *chi, int ng, int nw, cudaStream_t st);

// ---- stage (b), FP64 tensor cores (contract_f64.cu)
// One job = one chi block: chi[G][G'] += sum_p conj(M[p][G]) delta[p] M[p][G'] on upper tiles.
struct __align__(128) F64Job {
    CUtensorMap tm;       // M as doubles [P][2 ng], box {2 BT, 16}
    const double *delta;  // [P]
    double *chi;          // [ng][ng] complex
    int64_t P;
    int ng, ntile, ksplit, item_start;
};
cudaError_t launch_contract_f64_jobs(int bt, const F64Job *jobs, int njobs, int nitems, int grid, int *status,
                                     cudaStream_t st);
int contract_f64_bk();
size_t contract_f64_smem(int bt);

// ---- stage (b), split precision on BF16 tensor cores (ozaki.cu)
// sp[i] = sqrt(-delta[i])
cudaError_t launch_oz_sqrt(const double *delta, int64_t n, double *sp, cudaStream_t st);
// E[g] = column exponent of s_p M[p][g] over the chunk
cudaError_t launch_oz_colexp(const double2 *M, int64_t P, int ng, const double *sp, int *E, cudaStream_t st);
// A group of nw <= oz_group_w() frequencies at once (scales sp + w dstride): exponents E[w][ng],
// slices of frequency w at Z + w zstride (bf16 elements); M read once per pass for the group.
int oz_group_w();
cudaError_t launch_oz_split_multi(const double2 *M, int64_t P, int ng, const double *sp, int64_t dstride, int nw,
                                  int *E, int s, int64_t kpad, void *Z, int64_t zstride, cudaStream_t st);
// Z[i][j][p] bf16 slices, rows p in [P, kpad) zero
cudaError_t launch_oz_slice(const double2 *M, int64_t P, int ng, const double *sp, const int *E, int s,
                            int64_t kpad, void *Z, cudaStream_t st);
// One job = the split contraction of one chunk into one chi block (upper tiles).
struct __align__(128) OzJob {
    CUtensorMap tmA, tmB; // slices [s][2 ng][kpad] bf16, boxes {64, 128} and {64, BN}
    const int *E;         // [ng] column exponents
    double *chi;          // [ng][ng] complex
    int ng, nk, s, ntiles, item_start;
    int kb0;              // first K-step of this job (jobs may split K; the epilogue adds)
    // general product (launch_oz_gemm_general): out[rows_a][rows_b] real (complex pairs)
    // += A B with A slices by row (exponents E[rows_a]) and B^T slices by row (exponents
    // E2[rows_b / 2])
    const int *E2;
    double *out;
    int64_t ldo;
    int rows_a, rows_b;
};
// stages: TMA ring depth, 4 (default) or 2 (room on the SM for pair-kernel blocks alongside)
cudaError_t launch_oz_gemm_jobs(int bn, const OzJob *jobs, int njobs, int nitems, int grid, int *status,
                                cudaStream_t st, int stages = 4);
int oz_tiles(int ng, int bn);
int oz_pick_bn(int ng, int nsm); // tile width (240 or 256) by the wave count, without a tuned value
// General split product: Y[rows][nout] (complex, row-major, overwritten) = A[rows][ka] B[ka][nout]
// (complex, row-major), A split by rows and B by columns into s six-bit BF16 slices.
// ZA: s * rows * kpad bf16, ZB: s * 2 nout * kpad bf16, EA: rows ints, EB: nout ints,
// kpad = ka rounded up to a multiple of 32 complex (64 real) entries.
// conj: split the rows of conj(A) / the columns of conj(B).  B[g][b] is read at B[g sk + b sj]
// (sk = nout, sj = 1: row-major [ka][nout]; sk = 1, sj = ka: a row-major [nout][ka] transpose).
cudaError_t launch_oz_split_rows(const double2 *A, int64_t rows, int ka, int s, int64_t kpad, void *ZA, int *EA,
                                 cudaStream_t st, bool conj = false);
cudaError_t launch_oz_split_cols(const double2 *B, int ka, int nout, int64_t sk, int64_t sj, bool conj, int s,
                                 int64_t kpad, void *ZB, int *EB, cudaStream_t st);
// Plasmon-pole prep. step straight into row slices of P^T (the layout of launch_oz_split_rows with
// rows = ka = ng): P[g][c] = A[g][c] / (d - sgn wt[g][c]) in two-float arithmetic, At / Wt = A
// and wt transposed [c][g] as two-float (hi, lo) pairs (gpp_setup_tf), for cnt <= kGppMaxE
// energies d[0..cnt) (host) at once: slices of energy j at Z + j zstride (bf16 elements),
// exponents at E + j ng.
constexpr int kGppMaxE = 16;
struct GppEnergies {
    double d[kGppMaxE];
};
cudaError_t launch_gpp_prep_split(const float4 *At, const float4 *Wt, int ng, const double *d, int cnt, float sgn,
                                  int s, int64_t kpad, int64_t zstride, void *Z, int *E, cudaStream_t st);
cudaError_t launch_oz_gemm_general(int bn, const OzJob *jobs, int njobs, int nitems, int grid, int *status,
                                   cudaStream_t st);
size_t oz_smem_bytes(int bn, int stages = 4);
int oz_box_rows_a();
int oz_box_k();

// ---- adjoint of L = Re Tr(W chi) (adjoint.cu)
cudaError_t launch_zgemm(const double2 *A, const double2 *B, double2 *C, int64_t mr, int kd, int nc, cudaStream_t st);
// C (+)= op(A) op(B): conj_a takes conj(A); trans_b reads B as its transpose, row-major [nc][kd];
// accumulate adds into C.  Built for (conj_a), (trans_b, accumulate) and the plain product.
cudaError_t launch_zgemm_ex(const double2 *A, const double2 *B, double2 *C, int64_t mr, int kd, int nc, bool conj_a,
                            bool trans_b, bool accumulate, cudaStream_t st);
// ---- plasmon-pole self-energy, prep. step (sigma.cu)
// A[g][c] = v[c] Omega2[g][c] / (2 wt[g][c]) in FP64, stored [g][c]
cudaError_t launch_gpp_setup(const double2 *omega2, const double2 *wtilde, const double *vcoul, int ng, double2 *A,
                             cudaStream_t st);
// the same A and wt, transposed [c][g], as two-float (hi, lo) pairs for the split path
cudaError_t launch_gpp_setup_tf(const double2 *omega2, const double2 *wtilde, const double *vcoul, int ng, float4 *At,
                                float4 *Wt, cudaStream_t st);
// sigma[e][l][m] = ST[m][e nsig + l] (ST accumulated transposed by the split path)
cudaError_t launch_gpp_untranspose(const double2 *ST, int ne, int nsig, double2 *sigma, cudaStream_t st);
// P[g][c] = A[g][c] / (d - sgn wt[g][c]) (FP64, stored)
cudaError_t launch_gpp_prep_f64(const double2 *A, const double2 *wtilde, int ng, double d, double sgn, double2 *P,
                                cudaStream_t st);
cudaError_t launch_adj_rows(const double2 *M, double2 *Y, int64_t P, int ng, int nc, int64_t p0, const double *ev,
                            const double *ec, double w, double *L, double *dEv, double *dEc, cudaStream_t st);
// twofloat: the back-projection in two-float arithmetic (band grids in two-float form), H then
// holds float4 (hi, lo) pairs and launch_adj_products reads it that way and accumulates pbv / pbc
// in that form too (launch_tf_to_f64 converts them before the band adjoint), and Gb's rows are
// overwritten with conj(g_p) in two-float form; else FP64, Gb read only
cudaError_t launch_adj_pair(double2 *Gb, int64_t P, const PairPlan &pp, const int *cell_start,
                            const int *cell_g, int ncell, double2 *H, bool twofloat, cudaStream_t st);
// two-float (float4 hi/lo pairs) to complex128, in place, n points
cudaError_t launch_tf_to_f64(void *x, int64_t n, cudaStream_t st);
cudaError_t launch_adj_products(const void *psiv, const void *psic, int v0, int nvc, int nc, const double2 *H,
                                int64_t nr, bool tf, double2 *pbv, double2 *pbc, cudaStream_t st);
cudaError_t launch_band_adjoint(double2 *pb, int nb, const int n[3], const FftAxis ax[3], const int32_t *gofs,
                                int ngpsi, double2 *dc, cudaStream_t st);

} // namespace gw
