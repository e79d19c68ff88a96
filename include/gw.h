/*
 * gw.h -- C ABI of libgw, the GB300 (sm_103a) hot path of the Matsubara-time
 * GW cycle of Chu et al., "All-electron self-consistent GW in the
 * Matsubara-time domain" (arXiv:1602.02313), Sec. III.B.
 *
 * Conventions (all entry points):
 *  - The caller owns every buffer. Array arguments are DEVICE pointers unless
 *    marked "host". Nothing is returned to the host inside the per-q chain.
 *  - Complex numbers are interleaved (re, im) FP64 pairs ("cplx" below).
 *    Arrays are row-major with the shape given in brackets.
 *  - Energies are in Ha and measured from the chemical potential mu = 0
 *    (Sec. III.B.1); beta is in 1/Ha.
 *  - Band-pair convention: M[q][k][I][a][b] = M^I_ab(k, q) with band a at
 *    k - q and band b at k. This is Eq. (mmatrix) with k relabelled k -> k - q,
 *    so the same tensor serves Eq. (irpol) (P) and Eq. (sigc) (Sigma^c).
 *  - Calls are asynchronous and ordered on the stream given to gw_create.
 *    Argument errors are returned immediately (GW_EINVAL); a CUDA launch
 *    error is returned as GW_ECUDA; errors of asynchronous work surface at the
 *    next call or at gw_sync. gw_last_error() gives a readable message.
 *  - There is no CPU fallback: every step runs in libgw's CUDA kernels.
 *  - A context must not be used from two host threads at once.
 */
#ifndef GW_H
#define GW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gw_ctx gw_ctx;

typedef enum {
  GW_OK = 0,
  GW_EINVAL = -1,        /* bad argument (null pointer, size out of range) */
  GW_ENOMEM = -2,        /* device allocation failed */
  GW_ECUDA = -3,         /* CUDA runtime error */
  GW_ESINGULAR = -4,     /* zero pivot in a dielectric solve (see info[]) */
  GW_ENOCONV = -5,       /* continuation / QP iteration did not converge (see info[]) */
  GW_ETIMEOUT = -6,      /* a bounded device-side wait ran out */
  GW_EUNSUPPORTED = -7   /* combination not built (e.g. precision for this size) */
} gw_status;

/* Arithmetic of the P and Sigma^c contractions. */
typedef enum {
  GW_FP64 = 0,    /* native FP64 (CUDA cores); the parity path */
  GW_FP16X2 = 1,  /* tcgen05 tensor cores: fp16 hi/lo split operands, 3 products, FP32 TMEM accumulation */
                  /* (value 2 is not used) */
  GW_F32X2 = 3,   /* float-float on the FP32 pipes: each value hi + lo in two FP32 (~44-bit significand) */
  GW_F32 = 4      /* plain FP32 on the CUDA cores (gw_screen only) */
} gw_prec;

typedef enum { GW_BOSE = 0, GW_FERMI = 1 } gw_stat;

typedef enum {
  GW_TAU_TO_IW = 0,       /* tau -> sparse Matsubara set (nu_idx or w_idx) */
  GW_IW_TO_TAU = 1,       /* sparse Matsubara set -> tau */
  GW_TAU_TO_IW_CONT = 2   /* FERMI only: tau -> dense set w_n, n = 0 .. ncont-1 */
} gw_dir;

typedef enum { GW_PADE = 0, GW_CPE = 1 } gw_cont_method;

/* Discretisation (all host arrays, copied by gw_create). */
typedef struct {
  double beta;            /* inverse temperature, 1/Ha */
  int ntau;               /* number of tau nodes (even) */
  const double* tau;      /* host [ntau]: ascending in (0, beta), closed under tau -> beta - tau */
  int npole;              /* Lehmann basis size, 1 <= npole <= ntau */
  const double* poles;    /* host [npole]: real frequencies E_l of the basis exp(-E tau)/(1+exp(-beta E)) */
  int nnu;                /* bosonic sparse set size */
  const int* nu_idx;      /* host [nnu]: n >= 0, nu_n = 2 n pi / beta */
  int nw;                 /* fermionic sparse set size */
  const int* w_idx;       /* host [nw]: n >= 0, w_n = (2 n + 1) pi / beta */
  int ncont;              /* dense fermionic set n = 0 .. ncont-1 for continuation (<= 512) */
} gw_grid;

/* Synthetic crystal. */
typedef struct {
  uint64_t seed;          /* key of the Philox4x32-10 stream of M */
  int nk;                 /* k points (q runs over nq of them) */
  int nq;                 /* q points handled by this context */
  int nb;                 /* bands per k (<= 256) */
  int nocc;               /* occupied bands (used only for reporting) */
  int ni;                 /* product-basis size (multiple of 32, <= 1024) */
  double omega;           /* unit-cell volume Omega in 1/(Omega N_k) of Eqs. irpol, sigc */
  const int* kmq;         /* host [nq][nk]: index of k - q */
  const double* v;        /* host [nq][ni]: diagonal Coulomb v_I(q) > 0 */
  const double* M;        /* device cplx [nq][nk][ni][nb][nb], or NULL: libgw generates M
                             from seed (Philox4x32-10, counter = flat index of
                             (q0 + iq, k, I, a, b), Box-Muller, E|M|^2 = 1/nb) and keeps it
                             in its own HBM buffer */
  int q0;                 /* global index of this context's first q (for the generator
                             counter; 0 unless the q points are split over several contexts) */
  int m_mode;             /* with M == NULL: 0 = as 3 when all q take at most half of the free
                             device memory, else as 2; 1 = all q generated in gw_create;
                             2 = one q at a time, regenerated on first use by a call that needs
                             M[q] (a crystal whose M does not fit in HBM); 3 = all q kept, each
                             generated on an internal low-priority stream when the q before it
                             is first used (q = 0 at gw_create), so that generation overlaps
                             the contractions; calls on the context's stream wait for it */
} gw_system;

/* Create a context on `device`, ordered on the cudaStream_t `stream` (NULL =
 * legacy default stream). Builds the tau <-> Matsubara transform matrices
 * (Lehmann-basis least squares, formed in double-double arithmetic) and, when
 * sys->M is NULL, allocates nq*nk*ni*nb*nb*16 bytes of HBM and generates M.
 * Returns GW_EINVAL for inconsistent sizes, GW_ENOMEM if HBM runs out. */
gw_status gw_create(gw_ctx** ctx, const gw_grid* grid, const gw_system* sys, int device,
                    void* stream);
gw_status gw_destroy(gw_ctx* ctx);
/* Waits for the context's stream and reports errors of its asynchronous work: GW_ECUDA for a
 * CUDA error, GW_ETIMEOUT when a bounded device-side wait in a tensor-core contraction (the
 * pipeline barriers of k_pol_tc / k_sig_tc, see GW_TUNE_WAIT_CYCLES) ran out since the last
 * gw_sync: the kernel then stopped, let the copies and MMAs it had issued finish, freed its
 * tensor memory and returned, and the outputs of those calls are undefined. The error word is
 * cleared when it is reported, so the context stays usable. */
gw_status gw_sync(gw_ctx* ctx);
const char* gw_last_error(gw_ctx* ctx);

/* Green's function on the tau grid.
 * sigx, vxc, sigc_iw all NULL: reference G0_j(k|tau) = -exp(-eps tau)[1 - n_F(eps)]
 *   (Sec. III.B.1), evaluated without overflow; occ = n_F(eps) = G(0^-) = -G(beta^-).
 * otherwise: diagonal Dyson update (Eqs. dysongf, zxjk, zcjk) posed at the sparse
 *   fermionic set: G(i w) = 1/(i w - eps - sigx + vxc - sigc_iw(i w)); the pole
 *   1/(i w - eps~), eps~ = eps + sigx - vxc, is subtracted and added back exactly in tau.
 * eps [nk][nb]; sigx, vxc [nk][nb]; sigc_iw cplx [nk][nb][nw];
 * G_tau out [nk][nb][ntau]; occ out [nk][nb]. */
gw_status gw_green_tau(gw_ctx* ctx, const double* eps, const double* sigx, const double* vxc,
                       const double* sigc_iw, double* G_tau, double* occ);

/* Irreducible polarization of the iq-th q, Eq. (irpol):
 * P_II'(q|tau) = 1/(Omega N_k) sum_k sum_ab M^I_ab Q_ab(tau) conj(M^I'_ab),
 * Q_ab(tau) = G_b(k|tau) G_a(k-q|-tau), G(-tau) = -G(beta - tau) (Sec. II).
 * G_tau [nk][nb][ntau] (any G: G0 or dressed); P_tau out cplx [ntau][ni][ni] (Hermitian). */
gw_status gw_polarization(gw_ctx* ctx, int iq, const double* G_tau, gw_prec prec, double* P_tau);

/* The polarization of several crystals (one q each) in one persistent launch: job j is
 * gw_polarization(ctxs[j], iqs[j], G_tau[j], prec, P_tau[j]), with the same results bit for bit.
 * All work runs on ctxs[0]'s stream (order the other contexts' earlier work before it). Each job's
 * operand image and pair weights are built first; then one thread block per SM pulls work units
 * (job, K segment, strip, tau) from a device counter until all are taken, so that the units of
 * small crystals fill the GPU beside those of large ones (the batched heterogeneous workload);
 * then each job's partials are summed into its P. ctxs, iqs, G_tau, P_tau are HOST arrays of
 * njobs entries (G_tau[j], P_tau[j] device pointers as in gw_polarization). 1 <= njobs <= 16,
 * every context at most once and all on one device, else GW_EINVAL; prec GW_FP16X2 only, else
 * GW_EUNSUPPORTED. A device wait that runs out is reported by gw_sync(ctxs[0]). No host-device
 * copy: the call can be captured into a CUDA graph once every context has run one polarization. */
gw_status gw_polarization_many(int njobs, gw_ctx* const* ctxs, const int* iqs, const double* const* G_tau,
                               double* const* P_tau, gw_prec prec);

/* Imaginary time <-> Matsubara transforms (Eq. trans and its bosonic / inverse
 * counterparts), fixed matrices (built in extended precision, stored FP64) applied as
 * batched matvecs. prec: GW_FP64 (native FP64), or GW_F32X2 for the two bosonic
 * directions (float-float arithmetic, relative error ~1e-13; the mixed chain's choice);
 * anything else returns GW_EUNSUPPORTED.
 *  BOSE  TAU_TO_IW : in cplx [ntau][batch]        -> out cplx [nnu][batch]
 *  BOSE  IW_TO_TAU : in cplx [nnu][m][m] of a Hermitian-matrix function (batch = m)
 *                    -> out cplx [ntau][m][m]; uses W(-i nu) = W(i nu)^dagger
 *  FERMI TAU_TO_IW : in real [batch][ntau]        -> out cplx [batch][nw]
 *  FERMI TAU_TO_IW_CONT : in real [batch][ntau]   -> out cplx [batch][ncont]
 *  FERMI IW_TO_TAU : in cplx [batch][nw] of a real tau-function -> out real [batch][ntau] */
gw_status gw_tau_to_freq(gw_ctx* ctx, gw_stat stat, gw_dir dir, int64_t batch, const double* in,
                         gw_prec prec, double* out);

/* count independent transforms of gw_tau_to_freq in one call, their inputs and outputs stored
 * one after another (in [count][...in of one transform], out [count][...out of one]); the
 * bosonic directions run them in one grid (q points of a block of the chain), the fermionic
 * ones as one batch of count * batch rows. Results are those of count separate calls.
 * 1 <= count <= 65535, else GW_EINVAL. Float-float inputs are converted through a context
 * workspace in chunks of at most 2 GiB. */
gw_status gw_tau_to_freq_many(gw_ctx* ctx, gw_stat stat, gw_dir dir, int count, int64_t batch, const double* in,
                              gw_prec prec, double* out);

/* Screened interaction minus bare Coulomb, W~ = W - v (Sec. III.B.3), at the bosonic
 * sparse set, where Eq. (tildeW) is algebraic: Pi = v^1/2 P v^1/2, X = (1 - Pi)^-1 Pi,
 * W~ = v^1/2 X v^1/2, for the nqb q points iq0 .. iq0 + nqb - 1 at once. With ni a
 * multiple of 32 (every ni gw_create accepts; NI > 320 runs the pivot-row panels in
 * passes) X = (1 - Pi)^-1 - 1 from a blocked in-place Gauss-Jordan inversion; the
 * elimination of [1 - Pi | Pi] (GW_FP64 only, any ni) serves gw_screen_static. No pivoting:
 * 1 - Pi has Hermitian part >= 1.
 * prec: GW_FP64 (native FP64), GW_F32X2 (float-float arithmetic; relative error ~1e-12
 * per element) or GW_F32 (FP32 arithmetic, blocked inversion only; relative error of the
 * order of sqrt(ni) 6e-8 cond(1 - Pi), ~1e-6 at ni = 256); else GW_EUNSUPPORTED.
 * P_iv, Wt_iv cplx [nqb][nnu][ni][ni]; info out (device) [nqb][nnu]: 0, or j+1 for a
 * zero pivot at elimination step j (that system's output is then undefined).
 * Uses nqb * nnu * ni * 2 ni * 16 bytes of workspace that the context allocates
 * (and grows) on first use. */
gw_status gw_screen(gw_ctx* ctx, int iq0, int nqb, const double* P_iv, gw_prec prec, double* Wt_iv, int* info);

/* The paper's tau-domain form of Eq. (tildeW) (Sec. III.B.3, after Stan et al.), the
 * cross-check of the i nu route on small meshes: on a mesh tau_0 = 0 < tau_1 < ... < tau_M = beta
 * (npts = M + 1, e.g. the uniform power mesh of Sec. III.A) with the trapezoid increments
 * dtau_r = (tau_{r+1} - tau_{r-1}) / 2 (half the end intervals at r = 0 and M), solves
 *   sum_r sum_J [delta_IJ delta_pr - v_I P_IJ(tau_p - tau_r) dtau_r] W~_JJ'(tau_r) = v_I P_IJ'(tau_p) v_J'
 * for W~(tau_r), r = 0..M, v the context's Coulomb diagonal of its iq-th q.
 * tau [npts]: HOST array, strictly increasing, tau_0 = 0 (else GW_EINVAL).
 * P_pair cplx [npts][npts][ni][ni] (device): P_pair[p][r] = P(tau_p - tau_r) with the difference
 * taken modulo beta (bosonic; differences 0 and +-beta give P(0)).
 * Wt_tau out cplx [npts][ni][ni] (device); info (device int): 0, or k + 1 when elimination
 * step k found no non-zero pivot (the output is then undefined).
 * Gauss-Jordan elimination with partial pivoting in FP64 on the (npts ni) x (npts ni + ni)
 * augmented system, one launch per pivot; workspace 2 (npts ni)(npts ni + ni) 16 bytes, grown
 * on use. The increments are copied to the device synchronously before the call returns, so
 * the call cannot be captured into a CUDA graph. */
gw_status gw_screen_tau(gw_ctx* ctx, int iq, int npts, const double* tau, const double* P_pair, double* Wt_tau,
                        int* info);

/* The paper's tau-domain Dyson equation for the diagonal G (Sec. III.B.5, Eqs. dysongf, zxjk,
 * zcjk, dysong), the check of the i w update of gw_green_tau on small meshes. For each of nprob
 * states, Sigma^c given on a mesh tau_upm (HOST array of n_upm points, tau_0 = 0, last point
 * beta, every point a multiple of h = tau_1 - tau_0, as on the uniform power mesh) is carried
 * by a natural cubic spline to the uniform mesh t_i = i h, i = 0..n (n = beta / h), where
 *   sum_r [delta_pr - w_r Z(t_p, t_r)] G(t_r) = G0(t_p),
 *   Z(t, t2) = G0(t - t2) s + sum_l w_l G0(t - t_l) Sigma^c(t_l - t2),
 * w the trapezoid increments (h, h/2 at both ends); G0(tau) = -e^{-eps tau}(1 - n_F(eps)) and
 * Sigma^c are antiperiodic (f(d) = -f(d + beta) for d < 0; a zero difference takes the value
 * at 0+). eps, s [nprob] (device; s = Sigma^x + Sigma^H - Sigma_0 of the state);
 * sigc [nprob][n_upm] (device); G out [nprob][n + 1] (device, on the uniform mesh);
 * info [nprob] (device): 0, or k + 1 for a zero pivot at elimination step k (that state's G
 * is then not written). GW_EINVAL unless 3 <= n_upm <= 1024 and n + 1 <= 1024 and the mesh
 * is as described. FP64; one block per state (Gauss-Jordan with partial pivoting); workspace
 * (n + 1)(n + 2) 8 bytes per state, for chunks of states of at most 1 GiB. The mesh is copied
 * to the device synchronously before the call returns (not capturable in a CUDA graph). */
gw_status gw_dyson_tau(gw_ctx* ctx, int64_t nprob, int n_upm, const double* tau_upm, const double* eps,
                       const double* s, const double* sigc, double* G, int* info);

/* Crystal-symmetry reduction (Sec. III.C): the contribution of q' = R q to Sigma_n(k) equals the
 * contribution of q at R^-1 k, so a caller that computes P, W~ and gw_selfenergy for the
 * irreducible q points only, each into a zeroed buffer T, carries each one to its star with
 *   S[k][c] += sum_{r < nrep} T[kinv[r][k]][c],   c < ncol,
 * kinv [nrep][nk] (device int): index of R_r^-1 k on the mesh, one row per member R_r q of the
 * star; T, S [nk][ncol] (device; ncol = nb ntau for Sigma^c, nb for Sigma^x). Entries of kinv
 * outside [0, nk) are skipped. GW_EINVAL for nrep < 1 or ncol < 1. */
gw_status gw_sigma_star(gw_ctx* ctx, int nrep, const int* kinv, int64_t ncol, const double* T, double* S);

/* Off-diagonal self-energy of the iq-th q in the band basis (Eqs. sigc and sigx without the
 * diagonal approximation of Sec. III.B), ACCUMULATED:
 *   Sigma^c_nm(k|tau) += -1/(Omega N_k) sum_j G_j(k-q|tau) sum_IJ conj(M^I_jn) W~_IJ(tau) M^J_jm,
 *   Sigma^x_nm(k)     += -1/(Omega N_k) sum_j occ_j(k-q) sum_I v_I conj(M^I_jn) M^I_jm.
 * G_tau [nk][nb][ntau], occ [nk][nb] (may be NULL when Sx is), Wt_tau cplx [ntau][ni][ni];
 * S_tau cplx [nk][nb][nb][ntau]; Sx cplx [nk][nb][nb] (may be NULL). FP64 on the CUDA cores,
 * W~ a_j formed in chunks of rows so any ni fits; GW_EINVAL when the nb x nb accumulator of one
 * (k, tau) and 8 rows of W~ a_j do not fit in 200 KiB of shared memory (nb > 109). */
gw_status gw_selfenergy_offdiag(gw_ctx* ctx, int iq, const double* G_tau, const double* occ, const double* Wt_tau,
                                double* S_tau, double* Sx);

/* Dyson update of the full band matrix of G (Eq. dysonGF of Sec. II without the diagonal
 * approximation of Sec. III.B, whose off-diagonal form the paper leaves for later work), the
 * consumer of gw_selfenergy_offdiag. Posed at the sparse fermionic set like gw_green_tau:
 *   G(k|i w) = [i w - H~ - Sigma^c(k|i w)]^-1,   H~ = diag(eps) + Sx - vxc,
 * Sigma^c(i w) from Sc_tau by the fermionic forward transform (Eq. trans, complex-linear); the
 * tail (i w - H~)^-1 is subtracted and added back exactly in tau as U diag(G0(lambda, tau)) U^+
 * with H~ = U diag(lambda) U^+ (cyclic Jacobi on the device, Hermitian part of H~); the
 * remainder goes back to tau through the fermionic backward map of the real tau-functions
 * Re G_nm and Im G_nm.
 * eps [nk][nb]; Sx, vxc cplx [nk][nb][nb] (Hermitian; either may be NULL for zero);
 * Sc_tau cplx [nk][nb][nb][ntau] (NULL for zero); G_tau out cplx [nk][nb][nb][ntau];
 * occ out cplx [nk][nb][nb] = -G(beta^-); info out (device) int [nk]: 0, 1 when the eigensolver
 * did not reach 1e-15 relative off-diagonal norm in 40 sweeps (G is still written), or 2 + j
 * for a zero pivot at elimination step j of some frequency (that k's G and occ not written).
 * FP64 on the CUDA cores; nb <= 256 (else GW_EINVAL); workspace
 * ~ nk nb^2 (4 nw + 2) 16 bytes, grown on use. */
gw_status gw_dyson_matrix(gw_ctx* ctx, const double* eps, const double* Sx, const double* vxc, const double* Sc_tau,
                          double* G_tau, double* occ, int* info);

/* Allocation-free variant of gw_screen. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory at the time of the call, such as
 * code whose device memory was handed to another allocator at start-up, or a loop that must
 * not take the device-wide synchronisation a cudaMalloc can cause. It needs no context and
 * allocates nothing (no cudaMalloc / cudaFree, no allocating library call): its scratch is a
 * 128 MiB array compiled into libgw, which every GPU that loads the library keeps until the
 * process exits. The first call on a device looks up that array's device address (with the
 * device current) and caches it; make that first call before any stream capture.
 * All calls on a device share the one array and it keeps the last call's contents, so calls
 * that overlap on the GPU (different streams, or concurrent host threads) race; the solve
 * overwrites every scratch element it reads, so nothing needs clearing between calls.
 * Computes what gw_screen with GW_FP64 does (by elimination of [1 - Pi | Pi] in FP64; the
 * results agree to rounding), for nq q points at once:
 * sqrt_v (device) [nq][ni] = v_I(q)^(1/2); P_iv, Wt_iv cplx [nq][nnu][ni][ni]; info [nq][nnu].
 * Returns GW_EINVAL if one q point's systems (nnu * ni * 2 ni * 16 bytes) exceed 128 MiB,
 * GW_ECUDA on a launch error; runs on the cudaStream_t `stream` (NULL = legacy stream). */
gw_status gw_screen_static(int nq, int nnu, int ni, const double* sqrt_v, const double* P_iv, double* Wt_iv,
                           int* info, void* stream);

/* Contribution of the iq-th q to the self-energy, ACCUMULATED into the outputs:
 * Eq. (sigc): Sigc_n(k|tau) += -1/(Omega N_k) sum_j G_j(k-q|tau) a_jn^dagger W~(q|tau) a_jn,
 *             a_jn = M[q][k][:][j][n];
 * Eq. (sigx) in the product basis with diagonal v:
 *             Sigx_n(k) += -1/(Omega N_k) sum_j occ_j(k-q) sum_I v_I |M^I_jn|^2.
 * G_tau [nk][nb][ntau]; occ [nk][nb]; Wt_tau cplx [ntau][ni][ni] (Hermitian);
 * Sigc_tau [nk][nb][ntau] (real: W~(tau) Hermitian); Sigx [nk][nb] (may be NULL).
 * prec GW_FP64: both in FP64. GW_FP16X2: Sigc on the tensor cores, Sigx in
 * float-float on the FP32 pipes (relative error ~1e-12). */
gw_status gw_selfenergy(gw_ctx* ctx, int iq, const double* G_tau, const double* occ,
                        const double* Wt_tau, gw_prec prec, double* Sigc_tau, double* Sigx);

/* Analytic continuation and quasiparticle energies (Sec. III.B.6), one problem per (k, n).
 * sig_iw cplx [nprob][ncont]: Sigma^c at w_n, n = 0 .. ncont-1.
 * method GW_PADE: Vidberg-Serene continued fraction through the first npade points
 *   (npade = min(ncont, 64)).
 * method GW_CPE : continuous-pole expansion, Im Sigma piecewise linear on the real grid
 *   x_m (host [ngrid+2], hats on the ngrid interior nodes), b_m >= 0 fitted by
 *   Lawson-Hanson NNLS with a ridge lambda^2 |b|^2, lambda = ridge * ||A||_F.
 *   b0 (device [nprob][ngrid] or NULL) warm-starts the active set (learned seed).
 * eps, sigx, vxc [nprob]: QP root of E - eps - sigx + vxc - Re Sigma^c(E) nearest eps.
 * omega_real [nreal] (device); sig_real out cplx [nprob][nreal] at omega + i eta (eta = 1e-4);
 * e_qp out [nprob]; info out [nprob] (0 ok, 1 QP not converged, 2 NNLS iteration cap). */
gw_status gw_continue(gw_ctx* ctx, gw_cont_method method, int64_t nprob, const double* sig_iw,
                      const double* eps, const double* sigx, const double* vxc, int nreal,
                      const double* omega_real, double* sig_real, double* e_qp, int* info);

/* Real-axis grid of the continuous-pole expansion used by gw_continue(GW_CPE):
 * x host [ngrid + 2] ascending, ridge relative Tikhonov weight (>= 0). Must be
 * called before the first GW_CPE call; builds A^T A on the device. */
gw_status gw_cpe_setup(gw_ctx* ctx, int ngrid, const double* x, double ridge);
/* CPE coefficients of the last gw_continue(GW_CPE) call: b out [nprob][ngrid]. */
gw_status gw_cpe_coeffs(gw_ctx* ctx, double* b);

/* ---------------------------------------------------------------------------------------
 * Learned seed of the continuous-pole expansion (not in the paper). A multilayer perceptron
 * maps the normalised Matsubara self-energy of one (k, n) problem to non-negative pole weights
 * on the CPE grid; the weights warm-start the Lawson-Hanson fit of gw_continue(GW_CPE).
 * Training is unsupervised: L = (1/B) sum_b ||A b_hat_b - x_b||^2 with A the real-stacked CPE
 * kernel at the first nfit fermionic frequencies (gw_cpe_fit_matrix). All products run on the
 * tensor cores (fp16 operands, FP32 accumulation); weights are FP32 with fp16 copies.
 * ------------------------------------------------------------------------------------- */
typedef struct gw_mlp gw_mlp;

/* Network nin -> nh (nhidden GELU layers) -> nout (softplus). nin % 64 == 0, nh and nout % 128 == 0.
 * Weights drawn from a seeded generator; ordered on the cudaStream_t `stream`. */
gw_status gw_mlp_create(gw_mlp** mlp, int nin, int nh, int nhidden, int nout, uint64_t seed, int device,
                        void* stream);
gw_status gw_mlp_destroy(gw_mlp* mlp);
const char* gw_mlp_last_error(gw_mlp* mlp);
/* Number of parameters (per layer: W [out][in] row-major, then b [out]). */
int64_t gw_mlp_num_params(gw_mlp* mlp);
/* x (device) float [batch][nin] -> out (device) float [batch][nout]; batch % 128 == 0. */
gw_status gw_mlp_forward(gw_mlp* mlp, int64_t batch, const float* x, float* out);
/* Loss and gradients at the current weights (no update). x float [batch][nin] with nin = nx;
 * Acpe float [nx][nout]; loss (device, may be NULL) float [1]; grads (device, may be NULL)
 * float [num_params] in parameter order. */
gw_status gw_mlp_loss_grad(gw_mlp* mlp, int64_t batch, const float* x, int nx, const float* Acpe, float* loss,
                           float* grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr; loss as above. */
gw_status gw_mlp_train_step(gw_mlp* mlp, int64_t batch, const float* x, int nx, const float* Acpe, float lr,
                            float* loss);
/* Waits for the network's stream; GW_ETIMEOUT when a bounded wait of its tensor-core GEMM ran out
 * since the last sync (the results since then are undefined; the error is cleared). */
gw_status gw_mlp_sync(gw_mlp* mlp);
/* Host copies of the FP32 parameters in parameter order (float [num_params]); synchronises and
 * reports like gw_mlp_sync. */
gw_status gw_mlp_get_params(gw_mlp* mlp, float* params);
gw_status gw_mlp_set_params(gw_mlp* mlp, const float* params);

/* Network input from Sigma^c(i w): x float [nprob][2 nfit] = [Re, Im of the first nfit dense
 * frequencies] / scale, scale double [nprob] = max |component| (device arrays). */
gw_status gw_cpe_features(gw_ctx* ctx, int64_t nprob, const double* sig_iw, int nfit, float* x, double* scale);
/* A float [2 nfit][ngrid] (device): the CPE kernel at the first nfit dense frequencies (after gw_cpe_setup). */
gw_status gw_cpe_fit_matrix(gw_ctx* ctx, int nfit, float* A);
/* Warm start of the next gw_continue(GW_CPE) call with the same nprob: b0 = scale * bhat
 * (bhat float [nprob][ngrid], scale double [nprob], device). The active set starts at the
 * support of b0. Consumed by that call. */
gw_status gw_cpe_seed(gw_ctx* ctx, int64_t nprob, const float* bhat, const double* scale);
/* Lawson-Hanson outer iterations of the last gw_continue(GW_CPE) call: iters (device) int [nprob]. */
gw_status gw_cpe_iterations(gw_ctx* ctx, int* iters);

/* Matrix elements the context uses (for inspection and tests): copies
 * M[iq][k][:][:][:] for k in [k0, k0 + nk_copy) into out cplx [nk_copy][ni][nb][nb]. */
gw_status gw_copy_m(gw_ctx* ctx, int iq, int k0, int nk_copy, double* out);

/* Number of kernels libgw has launched on this context since gw_create (host counter). */
int64_t gw_launch_count(gw_ctx* ctx);

/* Per-kernel device timing. gw_kernel_timing(ctx, 1) discards earlier records and from then on
 * brackets every launch of the tensor-core contractions ("k_pol_tc", "k_sig_tc") and of the
 * blocked screening ("k_screen_inv") with CUDA events on the context's stream; 0 stops.
 * gw_kernel_time synchronises the stream and returns the summed device time (ms) and the
 * number of recorded launches of the named kernel. No device memory is allocated. */
gw_status gw_kernel_timing(gw_ctx* ctx, int enable);

/* Measured rates of the CUDA-core pipes on `device` (no context needed; runs two short
 * kernels of independent FMA chains): native FP64 and FP32 FMA throughput, TFLOP/s. A
 * float-float complex multiply-add (the mixed chain's screening and bosonic transforms) is 48
 * FP32-pipe operations, so fp32_tflops / 96 * 1e3 G/s is those kernels' ALU roofline.
 * Allocates 64 bytes. */
gw_status gw_measure_alu(int device, double* fp64_tflops, double* fp32_tflops);

/* Moves the context to another cudaStream_t (same device) for the calls that follow; work
 * already queued stays on the old stream (the caller orders the two). Lets one context serve as
 * a branch of a multi-stream CUDA graph. NULL = the legacy default stream. */
gw_status gw_set_stream(gw_ctx* ctx, void* stream);

/* Knobs of the tensor-core contractions.
 *  GW_TUNE_POL_SEG_CHUNKS: K chunks (32 pairs each) summed in one FP32 accumulator segment,
 *      1 .. 32 (default 32; fewer = more, smaller partials and a smaller accumulation error);
 *  GW_TUNE_POL_PART_MB: MiB of FP32 partial strips held at once (default 8192; the K segments
 *      run in passes beyond it), >= 1;
 *  GW_TUNE_WAIT_CYCLES: SM clock cycles a pipeline wait of k_pol_tc / k_sig_tc may take before it
 *      gives up and the launch reports GW_ETIMEOUT at the next gw_sync, 1e3 .. 2^40 (default 4e9,
 *      ~2 s at the GPU's top clock; a healthy wait takes microseconds);
 *  GW_TUNE_FAULT_STALL: fault injection for tests of that detector, 0 or 1: with 1, the
 *      MMA-issuing thread of every tensor-core contraction block first waits on a barrier that
 *      nothing arrives on, so the wait runs out after the wait budget (the GPU stays usable);
 *  GW_TUNE_POL_FORM: how the tensor-core polarization covers the Hermitian P(tau): 0 = by ni (the
 *      default: the real matrix E = Re P + Im P for ni <= 256, Re P and Im P over the Hermitian
 *      half above), 1 = always E, 2 = always Re P and Im P. Both give P within the same bound.
 * Out-of-range values return GW_EINVAL. Results stay within the tensor-core error bound. */
typedef enum {
  GW_TUNE_POL_SEG_CHUNKS = 0,
  GW_TUNE_POL_PART_MB = 1,
  GW_TUNE_WAIT_CYCLES = 2,
  GW_TUNE_FAULT_STALL = 3,
  GW_TUNE_POL_FORM = 4
} gw_tune;
gw_status gw_set_tuning(gw_ctx* ctx, gw_tune key, int64_t value);
gw_status gw_kernel_time(gw_ctx* ctx, const char* kernel, double* total_ms, int64_t* launches);

/* Host-only (no GPU needed): the transform matrices gw_create builds for `grid`,
 * written to host arrays (NULL entries skipped):
 * B_fwd cplx [nnu][ntau], F_fwd cplx [nw][ntau], F_cont cplx [ncont][ntau],
 * B_bwd real [ntau][2*nnu] (columns: Re-part weights, then Im-part weights),
 * F_bwd real [ntau][2*nw]. Returns GW_EINVAL for an inconsistent grid. */
gw_status gw_transform_matrices(const gw_grid* grid, double* B_fwd, double* F_fwd, double* F_cont,
                                double* B_bwd, double* F_bwd);

#ifdef __cplusplus
}
#endif

#endif /* GW_H */
