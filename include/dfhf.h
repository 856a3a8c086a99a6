/*
 * dfhf.h -- C ABI of the GB300 density-fitted Hartree-Fock library (libdfhf.so): restricted Hartree-Fock,
 * with unrestricted and restricted open-shell runs on the same builders.
 *
 * What the library computes (paper, arXiv:1707.03771):
 *   - every mean-field algorithm rests on density fitting (section "Program features");
 *   - the three-index tensor I_{gamma,rs} is held in memory (section "Density fitting utilities");
 *   - its operations, eqs. (1)-(3): index transformation (eq. 1), contraction of two fitted objects
 *     into a matrix (eq. 2, first form) and contraction with a density matrix (eq. 3, first two forms);
 *   - integrals are built from shell objects, the nuclear attraction also from the molecule
 *     (section "Molecular integrals").
 * Here: I = B_{P,mu nu} = sum_Q (L^-1)_{PQ} (Q|mu nu) with (P|Q) = L L^T (eq. 1, third form, M' = L^-1),
 *   gamma_P = sum B_{P,mu nu} D_{mu nu}, J = sum_P gamma_P B_P           (eq. 3, first and second forms)
 *   Y_{P,mu i} = sum_nu B_{P,mu nu} C_{nu i}, K = sum_{P,i} Y Y^T        (eq. 1 first form, eq. 2 first form)
 *   F = H + J - K, E = 1/2 tr(D(H + F)) + E_nuc, D = 2 C_occ C_occ^T    (RHF, section "Standard algorithms").
 * K as defined here is the exchange of the occupied orbitals (half the exchange matrix of D).
 *
 * Conventions (all functions):
 *   - Units: bohr and hartree. Shells are uncontracted real-solid-harmonic Gaussians, normalised to
 *     unit self-overlap; functions are ordered by shell, and within a shell m = -l..l.
 *   - Matrices are dense row-major doubles; symmetric inputs must be symmetric.
 *   - Host pointers are owned by the caller and only read/written during the call.
 *   - Device memory is owned by the handle and released by df_free.
 *   - Return value: DF_OK (0) or a negative DF_E* code; df_strerror gives its text, and
 *     df_last_error gives the detail of the last failure on that handle. No C++ exception crosses
 *     this interface.
 *   - One GPU: every call runs on the device that was current at df_init, on the handle's stream.
 *   - Host threads: calls on one handle must not overlap (one thread at a time per handle; the handle's
 *     buffers, stream and solver state are not locked). Calls on different handles may run concurrently
 *     from several threads: the process-wide state (the Rys root table, the autotuner's tile choices, the
 *     tensor-map encoder entry point, the atomic factors of the SAD guess) is guarded by mutexes, and each handle owns its stream, its cuSOLVER
 *     handle and its device buffers. The one shared device buffer is df_coulomb_noalloc's scratch (see
 *     there). scf_run_batch drives many handles from the calling thread alone.
 */
#ifndef DFHF_H
#define DFHF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DF_OK 0
#define DF_E_ARG (-1)        /* invalid argument (bad shell, l out of range, null pointer, size) */
#define DF_E_NOMEM (-2)      /* device allocation failed (e.g. B does not fit in HBM) */
#define DF_E_CUDA (-3)       /* CUDA runtime or cuSOLVER error */
#define DF_E_NOTCONV (-4)    /* SCF did not converge in max_iter iterations */
#define DF_E_STATE (-5)      /* call out of order (e.g. df_jk before df_build_B) */
#define DF_E_NUMERIC (-6)    /* metric not positive definite, singular DIIS, NaN */
#define DF_E_TIMEOUT (-7)    /* a device-side wait exceeded its iteration bound */

#define DF_LMAX_ORB 2        /* orbital shells: s, p, d */
#define DF_LMAX_AUX 3        /* auxiliary shells: s, p, d, f */

typedef struct { double xyz[3]; int Z; } df_atom;

/* One uncontracted shell. `center` is used as given (auxiliary shells may sit off the atoms);
 * `atom` is informational. exponent > 0, 0 <= l <= DF_LMAX_ORB (orbital) / DF_LMAX_AUX (aux). */
typedef struct { int atom; int l; double exponent; double center[3]; } df_shell;

/* Precision of the K contraction (paper silent; the split form is this library's design). */
#define DF_PREC_FP64 0       /* every step in FP64 */
#define DF_PREC_SPLIT 1      /* K from split BF16 slices on tensor cores, exact FP32 chunk sums, float-float sum */

#define DF_GUESS_CORE 0      /* core-Hamiltonian guess */
#define DF_GUESS_SAD 1       /* superposition of atomic densities (df_sad_density): the first Fock matrix is
                                built from that density itself */
#define DF_GUESS_SPIN 2      /* scf_run_uhf only: the natural orbitals of the spin densities of the handle's last
                                scf_run_uhf / scf_run_rohf (e.g. UHF from the ROHF solution) */

typedef struct {
    double conv_E;           /* |E_n - E_{n-1}| threshold (hartree), e.g. 1e-10 */
    double conv_err;         /* max |X^T (F D S - S D F) X| threshold, e.g. 1e-7 */
    int max_iter;            /* iteration cap */
    int diis_size;           /* Pulay subspace (<= 16) */
    int guess;               /* DF_GUESS_CORE or DF_GUESS_SAD (DF_GUESS_SPIN for scf_run_uhf; else DF_E_ARG);
                                scf_run_guess's D0 takes precedence */
    int precision;           /* DF_PREC_* */
    int slices;              /* BF16 slices per operand for DF_PREC_SPLIT (2..5) in early iterations;
                                once max|e| < 1e-4 the exchange is built with 5 slices, and the SCF
                                converges only on those builds */
    int incremental;         /* 1: late iterations (split: from the 5-slice ramp; FP64: once max|e| < 1e-4)
                                build K = K[D_ref] + K[D - D_ref], the change factorised exactly from the
                                occupied orbitals of both densities (QR of [C, C_ref], 2 nocc x 2 nocc
                                eigenproblem) and built at 3 slices; D_ref is rebuilt in full every 8
                                iterations. 0: every iteration builds K in full. */
    double screen_tau;       /* Schwarz screening threshold: validated (>= 0, else DF_E_ARG) but not
                                applied; every shell triple is computed (the FP64 parity bar needs 0) */
    int approx_diag;         /* 1: late iterations (max|e| < 1e-4) rotate the previous orbitals by
                                kappa_ia = F'_ia / (eps_a - eps_i) (approximate diagonalisation, Stewart,
                                Csaszar and Pulay 1982) instead of a full eigensolve; every 8th late
                                iteration diagonalises in full. The full eigensolves then run in FP32 and
                                are refined against the FP64 Fock matrix by one such rotation (and the
                                virtual orbitals projected out of the occupied space); the reported
                                orbitals and energies come from one FP64 eigensolve at the end. The result
                                is unchanged (convergence is tested on the exact commutator). 0: full FP64
                                eigensolve every iteration. */
} df_options;

typedef struct {
    double energy;           /* total RHF energy */
    double e_nuc;            /* nuclear repulsion */
    double e_one;            /* tr(D H) */
    double e_coul;           /* 1/2 tr(D J) */
    double e_exch;           /* -1/2 tr(D K) */
    double last_dE;
    double last_err;
    int iterations;
    int converged;
    int status;              /* DF_OK or DF_E_NOTCONV / DF_E_NUMERIC */
    int n_dropped;           /* orbitals removed by canonical orthogonalisation */
    int ramp_iteration;      /* split mode: first iteration built with 5 slices (0 if never) */
    int incremental_builds;  /* iterations whose K was K[D_ref] + K[D - D_ref] (options.incremental) */
    int approx_steps;        /* Roothaan steps taken by approximate diagonalisation (options.approx_diag) */
    double t_build_s;        /* df_build_B time within this call (0 if B was already built) */
    double t_iter_s;         /* total SCF iteration time */
    double t_jk_s;           /* time in J/K builds */
    double t_total_s;
    double s2;               /* <S^2> of the determinant (scf_run_uhf; 0 for RHF) */
    int graph_launches;      /* iteration parts launched as captured CUDA graphs (the J/K build and the Fock,
                                energy and DIIS-error part are captured per kind of step on its second
                                occurrence and replayed; DFHF_SCF_GRAPHS=0 launches every kernel directly) */
} df_result;

typedef struct df_handle df_handle;

/* Create a handle: copies atoms and shells, validates them, uploads shell tables and computes the
 * one-electron matrices S, T, V and the Coulomb metric (P|Q) on the GPU.
 * natom >= 1; nbasis_sh, naux_sh >= 1; charge must leave an even electron count (closed shell).
 * Returns DF_E_ARG for invalid shells (exponent <= 0, l out of range) or an odd electron count. */
int df_init(const df_atom* atoms, int natom, const df_shell* basis, int nbasis_sh,
            const df_shell* aux, int naux_sh, int charge, df_handle** out);

/* As df_init, but any electron count >= 1 is accepted (open-shell systems for scf_run_uhf). A handle with an
 * odd electron count is refused by the restricted entry points (scf_run, scf_run_guess, scf_run_batch:
 * DF_E_STATE); its nocc is ceil(N / 2). */
int df_init_open(const df_atom* atoms, int natom, const df_shell* basis, int nbasis_sh,
                 const df_shell* aux, int naux_sh, int charge, df_handle** out);

/* Sizes: n orbital functions, naux auxiliary functions, nocc doubly occupied orbitals, and the
 * length of one packed row of B (doubles). Any pointer may be NULL. */
int df_sizes(const df_handle* h, int* n, int* naux, int* nocc, long long* packed_row);

/* Three-centre integrals (P|mu nu) per angular-momentum class by Rys quadrature (paper, section
 * "Molecular integrals"), metric Cholesky (P|Q) = L L^T and whitening B = L^-1 (Q|mu nu) (eq. 1, third
 * form, M' = L^-1), stored packed (mu >= nu tiles) and kept in HBM (section "Density fitting utilities").
 * L^-1 is formed once in FP64; the whitening applies it as a 7-slice split-precision product.
 * Returns DF_E_NOMEM if the packed tensors do not fit; DF_E_NUMERIC if (P|Q) is not positive definite.
 * screen_tau as in df_options (must be >= 0; every triple is computed). keep_3c = 1 keeps the unwhitened tensor
 * for df_get_rows (needs twice the memory). */
int df_build_B(df_handle* h, double screen_tau, int keep_3c);

/* How the whitening B = L^-1 (Q|mu nu) is applied (the metric factor and its inverse are FP64 either way). */
#define DF_WHITEN_SPLIT 0    /* 7-slice split-precision product on the tensor cores (df_build_B's choice) */
#define DF_WHITEN_FP64 1     /* FP64 product on the FP64 pipe: slower (about 20 s at n = 1600, naux = 4384)
                                but FP64 end to end; scf_run builds B this way for DF_PREC_FP64 */

/* df_build_B with the whitening chosen (DF_WHITEN_*); a different value gives DF_E_ARG. Rebuilding B
 * drops the split-precision slices cut from the previous B. */
int df_build_B_ex(df_handle* h, double screen_tau, int keep_3c, int whitening);

/* B for n molecules (distinct handles on one device; the batched form of df_build_B_ex, the paper has no
 * counterpart): the three-centre integrals of all of them run as one persistent launch per angular-momentum
 * class over a global queue of (molecule, block of 128 shell pairs, block of 8 auxiliary shells) work items,
 * then each molecule's metric factor, inverse and whitening follow on its own stream. The integrals are
 * those of df_build_B to rounding (the same per-triple code in another kernel). Every handle needs room for its integrals at once. Returns the first failure
 * (each handle's df_last_error holds it); handles left without B are reset. */
int df_build_B_batch(df_handle** hs, int n, double screen_tau, int keep_3c, int whitening);

/* Coulomb and exchange matrices (paper eq. 3, first two forms, and eqs. 1-2, first forms) for density
 * D (n x n, symmetric) and occupied coefficients C_occ (n x nocc, row-major: C_occ[mu * nocc + i]):
 *   J = sum_P gamma_P B_P with gamma_P = sum B_{P,mu nu} D_{mu nu};  K = sum_{P,i} Y Y^T.
 * J and K are n x n outputs. device_ptrs = 1: all four are device pointers (on the handle's device);
 * 0: host pointers, copied in and out inside the call. precision: DF_PREC_FP64 or DF_PREC_SPLIT
 * (slices as in df_options). Requires df_build_B. */
int df_jk(df_handle* h, const double* D, const double* C_occ, int nocc, double* J, double* K,
          int device_ptrs, int precision, int slices);   /* slices: 2..5 for DF_PREC_SPLIT */

/* Full RHF SCF (paper, section "Standard algorithms": the Fock builder uses density fitting) from the
 * guess options.guess names; builds B first if needed (screen_tau from opts; DF_WHITEN_FP64 for
 * DF_PREC_FP64, DF_WHITEN_SPLIT for DF_PREC_SPLIT).
 * Results in *out; returns out->status. */
int scf_run(df_handle* h, const df_options* opts, df_result* out);

/* Batched SCF: nmol independent molecules (distinct handles on one device) solved together. Handles
 * without B get their three-centre integrals from one grouped launch per class (as df_build_B_batch) before
 * the iterations start; each molecule's metric factor and whitening run when it starts. Each
 * molecule's iteration is enqueued on its own stream; one host thread polls the molecules' completion
 * events and advances whichever has finished (convergence test, DIIS, orbital step, next iteration),
 * starting one more molecule per pass, so kernels of different molecules overlap on the GPU. B is built
 * first for handles that lack it. out[i] receives molecule i's result; the return value is DF_OK if all
 * converged, else the first failing status. */
int scf_run_batch(df_handle** hs, int nmol, const df_options* opts, df_result* out);

/* Superposition of atomic densities (the initial guess the SCF takes with options.guess = DF_GUESS_SAD; the
 * paper names no guess): every element gets a spherically averaged, fractional-occupation restricted
 * DF-HF of the neutral atom in the shells the molecule assigns to that atom (df_shell.atom, which must name
 * the atom for this guess): Aufbau occupations in which degenerate orbitals share their electrons equally,
 * F = H + J[D] - K with K the exchange of the occupied orbitals weighted by sqrt(n_i / 2), converged to
 * |dE| < 1e-11 Eh and max|X^T(FDS - SDF)X| < 1e-9 on the GPU. D0 (host, n x n) receives the block-diagonal
 * assembly of the atoms' densities, scaled to tr(D0 S) = N electrons. Atomic results are kept for the
 * process per element and shell set. DF_E_ARG if an atom with orbital shells has no auxiliary shells;
 * DF_E_NUMERIC if an atomic SCF does not converge. */
int df_sad_density(df_handle* h, double* D0);

/* Unrestricted Hartree-Fock with nalpha and nbeta electrons (paper, section "Program features", "Standard
 * algorithms": UHF on the density-fitted Fock builder): spin densities D_s = C_s C_s^T, J from D_a + D_b,
 * K_s = sum_{P, i in s} Y Y^T from each spin's occupied orbitals (FP64, or split precision: 3 slices until
 * max|e| < 1e-4, then 5, converging only on the 5-slice builds), F_s = H + J - K_s,
 * E = 1/2 tr(D_a(H + F_a)) + 1/2 tr(D_b(H + F_b)) + E_nuc, Pulay DIIS over the pair of orthogonal-basis Fock
 * matrices with errors X^T(F_s D_s S - S D_s F_s)X, core-Hamiltonian start for both spins, convergence as
 * scf_run on the larger of the two errors. out->s2 = <S^2>. Requires nalpha >= nbeta >= 0 and
 * nalpha + nbeta = electron count (DF_E_ARG otherwise); options.guess DF_GUESS_CORE, or DF_GUESS_SPIN to start
 * from the last open-shell run's spin densities (DF_E_STATE if the handle has none); incremental and
 * approx_diag 0. After the run df_get_matrix gives the total density (6) and the spin densities (12, 13). */
int scf_run_uhf(df_handle* h, const df_options* opts, int nalpha, int nbeta, df_result* out);

/* Restricted open-shell Hartree-Fock (same section of the paper: ROHF on the density-fitted Fock builder):
 * one orbital set, nbeta closed, nalpha - nbeta open, D_a / D_b from the first nalpha / nbeta orbitals,
 * F_s and E as in scf_run_uhf. Each step diagonalises the effective Fock matrix in the basis of the current
 * orbitals: closed-open blocks F_b, open-virtual blocks F_a, all other blocks (F_a + F_b)/2, plus
 * level_shift on the virtual and level_shift/2 on the open diagonal (the shift does not move the converged
 * energy; 0.5 Eh is a safe value, 0 can oscillate). DIIS over the effective matrix in the orthogonal basis
 * with its off-diagonal class blocks (proportional to the orbital gradient) as the error; convergence as
 * scf_run. out->s2 = S(S+1) up to rounding. Arguments, options and errors as scf_run_uhf; DF_E_ARG for a
 * negative or non-finite level_shift. */
int scf_run_rohf(df_handle* h, const df_options* opts, int nalpha, int nbeta, double level_shift,
                 df_result* out);

/* Density-fitted closed-shell MP2 correlation energy (paper, section "Program features": MP2 on the
 * density-fitting utilities; eq. 1 applied to both orbital indices, eq. 2 second form):
 *   B^P_ia = sum_{mu nu} C_mu i B_P,mu nu C_nu a, (ia|jb) = sum_P B^P_ia B^P_jb,
 *   E2 = sum_{ij ab} (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b), every orbital correlated,
 * in FP64 on the GPU from the handle's B. C: host, n x nmo row-major, column k = canonical orbital k in
 * ascending energy (the first nocc occupied; e.g. df_get_matrix 10 after scf_run, nmo = n - dropped); eps:
 * host, nmo orbital energies. Requires B (DF_E_STATE), 1 <= nocc < nmo <= n (DF_E_ARG). Device memory:
 * about 8 naux (np + 2 nmo) nocc bytes besides B. */
int df_mp2(df_handle* h, const double* C, const double* eps, int nmo, int nocc, double* e2);

/* ---- density-fitting object operations (paper, section "Density fitting utilities", eqs. 1-3) ----------
 * A df_tensor is a dense FP64 three-index object I[g][r][s] (g the auxiliary index, row-major) on the device
 * of the handle it was made with; every operation runs on that handle's stream (one thread at a time per
 * handle, as for the other calls) and returns when its result is complete. Host arrays are row-major and
 * owned by the caller. Free every tensor (df_tensor_free) before its handle. Dimensions that do not match
 * give DF_E_ARG; DF_E_NOMEM if a result does not fit. */
typedef struct df_tensor df_tensor;
/* A new object of naux x nr x ns, from host_init (naux nr ns doubles) or zeros if host_init is NULL. */
int df_tensor_create(df_handle* h, int naux, int nr, int ns, const double* host_init, df_tensor** out);
/* The handle's B as an object: naux x n x n, both triangles (DF_E_STATE before df_build_B). */
int df_tensor_from_B(df_handle* h, df_tensor** out);
int df_tensor_shape(const df_tensor* t, int* naux, int* nr, int* ns);
/* Copy the object to host (naux nr ns doubles). */
int df_tensor_get(const df_tensor* t, double* host);
void df_tensor_free(df_tensor* t);
/* Eq. 1, index transformations, into a new object:
 *   which 0: I'_{g,ts} = sum_r I_{g,rs} M_rt   (M: nr x nt; m_rows = nr, m_cols = nt)
 *   which 1: I'_{g,rt} = sum_s I_{g,rs} M_st   (M: ns x nt; m_rows = ns, m_cols = nt)
 *   which 2: I'_{g,rs} = sum_d M'_gd I_{d,rs}  (M': naux' x naux; m_rows = naux', m_cols = naux) */
int df_op_transform(const df_tensor* I, int which, const double* M, int m_rows, int m_cols, df_tensor** out);
/* Eq. 2, contractions of two objects into a host matrix `out`:
 *   which 0: M_st = sum_{g r} I_{g,rs} I2_{g,rt}       (I2: naux x nr x nt; out ns x nt)
 *   which 1: G_{rs,tu} = sum_g I_{g,rs} I2_{g,tu}      (I2: naux x nt x nu; out (nr ns) x (nt nu))
 *   which 2: M_gd = sum_{rs} I_{g,rs} I2_{d,rs}        (I2: naux2 x nr x ns; out naux x naux2) */
int df_op_contract(const df_tensor* I, const df_tensor* I2, int which, double* out);
/* Eq. 3: D_g = sum_rs I_{g,rs} M_rs (M: nr x ns; D: naux) and M_rs = sum_g D_g I_{g,rs}. */
int df_op_density_fit(const df_tensor* I, const double* M, double* D);
int df_op_density_back(const df_tensor* I, const double* D, double* M);
/* Eq. 3: I'_{g,tu} = sum_rs I_{g,rs} G_{rs,tu} (G: (nr ns) x (nt nu)), into a new naux x nt x nu object. */
int df_op_apply_four_index(const df_tensor* I, const double* G, int nt, int nu, df_tensor** out);

/* SCF from a guess density D0 (host, n x n, symmetric; NULL = core-Hamiltonian guess): the first
 * occupied orbitals are the nocc natural orbitals of D0 with the largest occupations in the S metric
 * (eigenvectors of X^T S D0 S X). Otherwise as scf_run. */
int scf_run_guess(df_handle* h, const df_options* opts, const double* D0, df_result* out);

/* ---- learned initial guess (the paper has no counterpart; the build's design) -------------------
 * Waters only: atoms as consecutive (O, H, H) triples, every water with the same basis. Each water's
 * frame: origin O, z along the H-O-H bisector, x along H1 - H2. A network maps DF_MLP_NFEAT
 * rotation-invariant features of the water's environment to the upper triangle of its diagonal density
 * block in that frame; blocks are rotated to the laboratory frame with real-solid-harmonic rotation
 * matrices and assembled block-diagonally. A second network adds the blocks between nearby waters
 * (df_mlp_guess_pairs). */
#define DF_MLP_NFEAT 57
typedef struct df_mlp df_mlp;

/* Fully connected network nin -> nhidden (x nlayers, ReLU) -> nout, FP32 weights, He-initialised from
 * `seed`; parameters live on the current device. */
int df_mlp_create(int nin, int nhidden, int nlayers, int nout, unsigned long long seed, df_mlp** out);
void df_mlp_free(df_mlp* m);
/* Number of parameters; layout per layer l: W_l (out x in, row-major) then b_l. */
long long df_mlp_nparams(const df_mlp* m);
/* Copy parameters to (set = 0) or from (set = 1, also resets the Adam state) a host float array. */
int df_mlp_params(df_mlp* m, float* host, int set);
/* Mean-squared-error loss over ns samples (X: ns x nin, Y: ns x nout, host) and its gradient with
 * respect to every parameter (host, nparams floats), by the GPU forward and backward kernels. */
int df_mlp_gradients(df_mlp* m, const float* X, const float* Y, int ns, float* grad, float* loss);
/* Adam training (lr, beta1 0.9, beta2 0.999) with shuffled minibatches (seeded); loss_history
 * (epochs floats, may be NULL) receives each epoch's mean batch loss. */
int df_mlp_train(df_mlp* m, const float* X, const float* Y, int ns, int epochs, int batch, float lr,
                 unsigned long long seed, float* loss_history);
/* Network outputs for ns samples (host arrays); bf16 = 1 runs BF16 weights and activations with FP32
 * accumulation, 0 the FP32 network. */
int df_mlp_predict(df_mlp* m, const float* X, int ns, int bf16, float* Y);
/* Features of every water (out: nwater x DF_MLP_NFEAT); returns DF_MLP_NFEAT or a DF_E_* code. */
int df_water_features(const df_atom* atoms, int natom, float* out);
/* Upper triangles of each water's diagonal block of D (host, n x n) in the water's frame
 * (out: nwater x nb(nb+1)/2 floats, nb = functions per water). */
int df_water_blocks(df_handle* h, const double* D, float* out);
/* D0 (host n x n) assembled from frame blocks (nwater x nb(nb+1)/2). */
int df_water_density(df_handle* h, const float* blocks, double* D0);
/* Learned D0 (host n x n) for the handle's water cluster with network m (bf16 = BF16 inference). */
int df_mlp_guess(df_handle* h, df_mlp* m, int bf16, double* D0);

/* Pair blocks. An ordered pair (w1, w2) of waters whose O atoms are at most `cutoff` bohr apart has
 * DF_MLP_NPFEAT features: the atoms of w2 in w1's frame relative to w1's O (/ 10 bohr), 5 bohr / r for the
 * nine atom pairs between the waters, a Gaussian expansion of the O-O distance. Its block is the
 * nb x nb block D[w1][w2] with both function sets rotated into w1's frame. */
#define DF_MLP_NPFEAT 26
/* The ordered pairs within cutoff (both orders, by w1 then w2): returns their number (or a DF_E_* code)
 * and writes up to max_pairs of them (pairs: 2 ints each) and their features (feats: DF_MLP_NPFEAT floats
 * each; may be NULL). max_pairs = 0 only counts. */
int df_water_pairs(const df_atom* atoms, int natom, double cutoff, int* pairs, int max_pairs, float* feats);
/* Frame blocks of the listed pairs of D (host n x n): out npairs x nb x nb floats, row-major. */
int df_pair_blocks(df_handle* h, const double* D, const int* pairs, int npairs, float* out);
/* Adds the laboratory-frame blocks of the listed pairs to D0 (host n x n) at [w1][w2] and, transposed, at
 * [w2][w1]; a pair listed in both orders contributes the mean of its two blocks. */
int df_pair_density(df_handle* h, const float* blocks, const int* pairs, int npairs, double* D0);
/* df_mlp_guess with network m, plus the pair blocks of every pair within cutoff predicted by network mp
 * (DF_MLP_NPFEAT inputs, nb * nb outputs). */
int df_mlp_guess_pairs(df_handle* h, df_mlp* m, df_mlp* mp, double cutoff, int bf16, double* D0);

/* Per-iteration record of the last scf_run: up to max_rows rows of 6 doubles
 * (iteration, energy, energy change, max|X^T(FDS - SDF)X|, exchange slices (0 = FP64), J/K build ms).
 * Returns the number of rows the run produced (which may exceed max_rows), or a negative DF_E_*. */
int df_scf_history(const df_handle* h, double* out, int max_rows);

/* Copy rows [p0, p0+count) of an auxiliary-indexed tensor, unpacked to (count, n, n):
 * which = 0: unwhitened (P|mu nu) (needs keep_3c), 1: whitened B. Host output. */
int df_get_rows(df_handle* h, int which, int p0, int count, double* out);

/* Copy a matrix to host: 0 S, 1 T, 2 V, 3 H, 4 metric (naux x naux), 5 L^-1 (naux x naux, lower),
 * 6 D, 7 F, 8 J, 9 K (last SCF iteration), 10 C (n x n, columns = orbitals), 11 orbital energies (n),
 * 12 and 13 the alpha and beta densities of the last scf_run_uhf. */
int df_get_matrix(df_handle* h, int which, double* out);

/* Rys quadrature nodes x (= t^2) and weights w for `count` arguments T (host arrays; x and w are
 * count x nroots): the Gauss rule of exp(-T x) x^{-1/2} dx / 2 on [0,1], whose moments are the Boys
 * functions, sum_i w_i x_i^k = F_k(T) for k < 2 nroots (paper, section "Molecular integrals": ERIs
 * by Rys quadrature). A test hook for the device routine the integral kernels use. 1 <= nroots <= 4. */
int df_rys(const double* T, int count, int nroots, double* x, double* w);

/* rint(v[i] 2^k[i]) with ties to even, for `count` values (host arrays; runs on the host, no GPU needed):
 * the integer T from which the split-precision kernels peel the BF16 slices of a value whose row has the
 * power of two e (k = 7 S - e; Ozaki, Ogita, Oishi and Rump's error-free splitting, the reading of the
 * paper's silent precision point). A test hook for the device routine, which takes the same code.
 * Returns DF_E_ARG for a negative count or a null array. */
int df_rint_pow2(const double* v, const int* k, long long count, long long* out);

/* Coulomb matrix J (n x n, device pointer) for the density D (n x n, device pointer) without any
 * device allocation; the paper has no counterpart. For callers that cannot call cudaMalloc (a host
 * application that owns all device memory through its own allocator, or a latency-critical loop that
 * cannot afford an allocation's synchronisation or failure). Same kernels and result as the J of
 * df_jk; the scratch (packed density, gamma, packed J) lives in a 48 MiB array inside the library,
 * which every GPU that loads the library holds until exit. df_init resolves the array's device address
 * for the handle's device (under lazy module loading this is what commits the array's memory) and
 * loads the Coulomb kernels, so this call itself allocates nothing; if df_init could not resolve the
 * address, this call returns DF_E_STATE with the reason in df_last_error. Requires df_build_B. Systems
 * needing more than 6,291,456 doubles of scratch (2 packed rows of B + naux; about n <= 2400) are
 * rejected with DF_E_ARG and a message in df_last_error. Work is enqueued on the handle's stream and the
 * call returns without waiting. All calls share the array: calls that overlap on the GPU race; calls
 * ordered on one stream are safe. Every failure sets df_last_error. */
int df_coulomb_noalloc(df_handle* h, const double* D, double* J);

/* Measured FP64 rate of the current device, the denominator of the FP64 kernels' roofline (the paper has no
 * counterpart): kind 0 times a DFMA loop (8 independent chains per thread), kind 1 an mma.sync m8n8k4 FP64
 * loop, each `iters` iterations over 4 CTAs of 256 threads per SM after a short warm-up launch. *tflops
 * receives 2 x multiply-adds / time, *ms (may be NULL) the timed launch's duration. Allocates a small sink
 * array. Returns DF_E_ARG for another kind, iters < 1 or a null tflops. */
int df_fp64_rate(int kind, long long iters, double* tflops, double* ms);

/* Host-side set-up without a GPU: builds and validates the Rys root/weight table (Gauss rules of the
 * Boys-function measure) and caches it as rys_table.bin beside the library (or at $DFHF_TABLE_CACHE).
 * Optional: the first integral call does the same. Returns DF_E_NUMERIC if the table fails its check. */
int df_prepare(void);

/* Stream used by the handle (a cudaStream_t); NULL selects the handle's own stream. */
int df_set_stream(df_handle* h, void* stream);

/* Per-phase device times of the last df_build_B / df_jk in milliseconds (CUDA events):
 * [0] 1e+metric, [1] three-centre ERI, [2] Cholesky+inverse, [3] whitening, [4] gamma, [5] J,
 * [6] Y half-transform (FP64), [7] K contraction (FP64), [8] whole split exchange, [9] split Y,
 * [10] split K contraction, [11] split slicing and reduction, [12] tile width of the tensor-core Y
 * kernel and [15] K tile width chosen by the autotuner, [13] K split (occupancy heuristic), [14] time
 * the process has spent autotuning, [16] kernel launches of the last J/K build, [17] metric Cholesky
 * factorisation and [18] inversion of its factor (both within [2]). Up to `count` (<= 20) values are
 * written. */
int df_timings(const df_handle* h, double* ms, int count);

void df_free(df_handle* h);
const char* df_strerror(int code);
const char* df_last_error(const df_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* DFHF_H */
