/*
 * rid.h -- C ABI of librid, a GB300 (sm_103a) implementation of the
 * Reinforced Dynamics (RiD) biased / restrained Langevin MD step run over many
 * walkers at once (RiD-kit, arXiv 2408.14070).
 *
 * Conventions for every entry point
 *   - Return value: an rid_status code.  On failure rid_last_error() returns a
 *     one-line message for the calling thread; no output is written unless
 *     the call returns RID_OK (results may be partially written on
 *     RID_ERR_NONFINITE, see below).
 *   - Arrays are dense, C order, in the element type named.  Positions and
 *     velocities are [walker][bead][xyz] float32.
 *   - `mem` says where ALL array arguments of that call live: RID_MEM_HOST
 *     (pageable or pinned host memory) or RID_MEM_DEVICE (device memory of
 *     the current CUDA device).  The library never keeps a caller pointer
 *     after the call returns (rid_submit is the one exception, see there).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Synchronous
 *     calls enqueue their work on it and return after it has completed.
 *   - The caller owns every array it passes.  The library owns the device
 *     copies of parameters and the resident walker state it allocates.
 *   - Units are reduced (kT, mass, length as given); angles are radians.
 *   - Objects are not thread-safe: one thread at a time per rid_system.
 */
#ifndef RID_H
#define RID_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RID_API __attribute__((visibility("default")))
#else
#define RID_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RID_OK = 0,
    RID_ERR_ARG = 1,        /* invalid argument (NULL, size, range)         */
    RID_ERR_OOM = 2,        /* device allocation failed / budget exceeded    */
    RID_ERR_CUDA = 3,       /* a CUDA runtime call failed                    */
    RID_ERR_NONFINITE = 4,  /* NaN/Inf appeared in positions or forces       */
    RID_ERR_TIMEOUT = 5,    /* a bounded wait expired                        */
    RID_NOT_READY = 6,      /* rid_poll: job not finished yet                */
    RID_ERR_STATE = 7,      /* call not valid in the object's current state  */
    RID_ERR_CANCELLED = 8   /* job was cancelled                              */
} rid_status;

enum { RID_MEM_HOST = 0, RID_MEM_DEVICE = 1 };

/* Arithmetic of the ensemble MLP.  Forces, CVs and the integrator are always
 * FP32; label running sums and energy reductions are FP64.
 *   RID_PREC_FP32  FP32 SIMT, every GEMM
 *   RID_PREC_BF16  tensor cores, BF16 operands, FP32 accumulation
 *   RID_PREC_FP8   tensor cores: the forward GEMMs with FP8 e4m3 operands
 *                  (weights scaled per matrix by amax/448, activations
 *                  tanh in [-1, 1] unscaled), the input-gradient GEMMs BF16;
 *                  FP32 accumulation throughout */
enum { RID_PREC_FP32 = 0, RID_PREC_BF16 = 1, RID_PREC_FP8 = 2 };

/* CV force applied in rid_eval_forces. */
enum { RID_BIAS_NONE = 0, RID_BIAS_ENSEMBLE = 1, RID_BIAS_RESTRAINT = 2 };

/*
 * A bead chain in implicit solvent (the stand-in for the paper's GROMACS
 * systems, Sec. "Exploration phase"), its torsion CVs (Sec. "CV selection",
 * torsion mode, periodic) and Langevin parameters.
 *   U = sum_bonds k_b/2 (r - r0)^2 + sum_angles k_a/2 (theta - theta0)^2
 *     + sum_dihedrals sum_{n=1..3} k_n (1 + cos(n phi - delta_n))
 *     + sum_{|i-j|>=3, r^2 < rc^2} [4 eps ((sig/r)^12 - (sig/r)^6) - U(rc)]
 * The LJ inclusion test r^2 < rc^2 is taken in FP32 with
 * r^2 = fma(dz, dz, fma(dy, dy, dx * dx)), d = x_j - x_i.  Torsions use the
 * IUPAC sign convention on [-pi, pi).
 */
typedef struct {
    int32_t n_beads;              /* N, 4 <= N <= 4096                          */
    int32_t n_cv;                 /* C, 1 <= C <= 128                           */
    int32_t output_freq;          /* trace stride in steps (>= 1)               */
    int32_t reserved0;            /* must be 0                                  */
    double mass, kT, dt, gamma;   /* bead mass, thermal energy, step, friction  */
    uint64_t seed;                /* Philox4x32-10 key                          */
    double bond_k, bond_r0;
    double angle_k, angle_theta0;
    double lj_eps, lj_sigma, lj_rc;
    const double* dihedral_k;     /* host [N-3][3]: k_1..k_3 per dihedral       */
    const double* dihedral_delta; /* host [N-3][3]: delta_1..delta_3            */
    const int32_t* cv_atoms;      /* host [C][4]: bead indices of each torsion  */
} rid_system_desc;

/*
 * Ensemble of M MLPs s -> A_i(s) (Sec. "Training phase": numb_models,
 * neurons, resnet).  Input u = (cos s_0, sin s_0, cos s_1, sin s_1, ...),
 * D = 2C; L hidden tanh layers of width H (residual h_l = h_{l-1} + tanh(.)
 * for l >= 2 when resnet != 0); scalar linear output.
 * Packed FP32 weights per model, models back to back:
 *   W_1[H][D], b_1[H], (W_l[H][H], b_l[H]) for l = 2..L, w_out[H], b_out[1].
 * Bias (Sec. "Development of the protocol"): U_bias = -Abar (the inverted
 * predicted PMF), applied with the switch sigma(eps) of the model deviation
 * eps = sqrt((1/M) sum_i |dA_i/ds - Fbar|^2):
 *   sigma = 1 (eps < trust_lo), 0 (eps >= trust_hi),
 *           (1 + cos(pi (eps - trust_lo)/(trust_hi - trust_lo)))/2 between
 * (trust_lvl_1 / trust_lvl_2, Sec. "Overall workflow setting"); CV force
 * F_s = sigma(eps) Fbar with Fbar = (1/M) sum_i dA_i/ds.
 */
typedef struct {
    int32_t n_models;             /* M, 1..16                                   */
    int32_t n_in;                 /* D, must equal 2 * n_cv                     */
    int32_t n_layers;             /* L, 1..8                                    */
    int32_t width;                /* H, 1..512 (padded inside to a multiple of  */
                                  /* 32 with zero units: the same function)     */
    int32_t resnet;               /* 0 / 1, at every precision                  */
    int32_t precision;            /* RID_PREC_*                                 */
    double trust_lo, trust_hi;    /* trust_lo < trust_hi                        */
    const float* weights;         /* host [M][P], copied by the call            */
} rid_ensemble_desc;

typedef struct rid_system rid_system;

/* Library identity and diagnostics. */
RID_API int rid_version(void);                       /* 10000 * major + 100 * minor   */
RID_API const char* rid_status_string(int status);
RID_API const char* rid_last_error(void);            /* thread-local, never NULL      */

/* Create a system on the current CUDA device.  Copies every array of desc.
 * Errors: RID_ERR_ARG (bad sizes / indices), RID_ERR_OOM, RID_ERR_CUDA. */
RID_API int rid_create_system(const rid_system_desc* desc, rid_system** out);
/* Release the system and all device memory it owns (NULL is accepted). */
RID_API int rid_destroy_system(rid_system* sys);

/* Set (or replace) the ensemble used by biased exploration.  Copies the
 * weights to device-resident FP32 (and BF16 for RID_PREC_BF16) tiles.
 * Errors: RID_ERR_ARG (shape mismatch with the system's C), RID_ERR_OOM. */
RID_API int rid_set_ensemble(rid_system* sys, const rid_ensemble_desc* desc);

/*
 * Biased exploration (Sec. "Exploration phase"): W walkers, n_steps BAOAB
 * Langevin steps each (one force evaluation per step), starting at global
 * step index step0 (the Philox counter; step0 + n_steps <= 2^32).  Without an
 * ensemble the run is unbiased MD.
 *   x0      [W][N][3]        starting positions
 *   v0      [W][N][3]|NULL   starting velocities; NULL draws Maxwell-Boltzmann
 *                            velocities from Philox stream 1 at step0
 *   cv_out  [W][T][C]|NULL   CVs after steps output_freq, 2 output_freq, ...
 *                            (T = n_steps / output_freq)
 *   eps_out [W][T]|NULL      model deviation at the same steps
 *   energy_out [W][T][3]|NULL  float64 (U_ff, -Abar, kinetic) at those steps
 *   x_out, v_out [W][N][3]|NULL  final state
 * Noise: counter (bead, walker, step, 0), key = seed; u = (word + 1/2) 2^-32;
 * Box-Muller on words (0,1) -> xi_x, xi_y and (2,3) -> xi_z.
 * Errors: RID_ERR_ARG, RID_ERR_OOM, RID_ERR_CUDA, RID_ERR_NONFINITE (the run
 * completed but some walker produced NaN/Inf; outputs are written).
 */
RID_API int rid_explore(rid_system* sys, int32_t n_walkers, const float* x0, const float* v0,
                uint64_t step0, int64_t n_steps, float* cv_out, float* eps_out,
                double* energy_out, float* x_out, float* v_out, int32_t mem, void* stream);

/*
 * Restrained-MD labelling (Sec. "Labeling phase", restrained method): R runs,
 * each with harmonic restraints U_r = sum_j kappa_j/2 wrap(s_j - s0_j)^2 on
 * every CV and no ensemble bias.  After n_equil steps every step contributes
 * d = wrap(s - s0) (wrap onto [-pi, pi)) to FP64 running sums on the device.
 *   s0, kappa [R][C] float64     restraint centres and force constants
 *   mf_out    [R][C] float64     mean force -kappa <d>
 *   se_out    [R][C] float64     standard error from n_blocks equal blocks:
 *                                kappa std_{ddof=1}(block means)/sqrt(B);
 *                                sample k of K goes to block floor(k B / K)
 *   std_out   [R][C] float64     population std of kappa d
 * Requires 2 <= n_blocks <= 256 and n_steps - n_equil >= n_blocks.
 */
RID_API int rid_label(rid_system* sys, int32_t n_runs, const float* x0, const float* v0,
              const double* s0, const double* kappa, uint64_t step0, int64_t n_steps,
              int64_t n_equil, int32_t n_blocks, double* mf_out, double* se_out, double* std_out,
              float* x_out, float* v_out, int32_t mem, void* stream);

/*
 * Constrained-MD labelling on distance CVs (Sec. "Labeling phase", constrained
 * method, Box 5: distance CVs only).  For each of R runs the C distances
 * r_j = |x_a - x_b| of `pairs` [C][2] (host int32; distinct beads, no bead in
 * two pairs) are held at d0 [R][C] (float64, > 0) by SHAKE / RATTLE inside the
 * BAOAB step (the system's dt, gamma, kT, mass and force field; no ensemble
 * bias, and the system's torsion CVs play no part).  The start x0 is moved
 * onto the constraints (each pair symmetrically along its own axis).  After
 * n_equil steps every step samples the mean force along each distance,
 *   F_j = -(f_a - f_b) . u_j / 2 - 2 kT / d0_j   (f: force-field forces,
 *   u_j = (x_a - x_b) / d0_j; the free energy includes the r^2 of the shell),
 * and mf_out / se_out / std_out [R][C] receive its mean, the standard error
 * from n_blocks equal blocks and its population std.  Noise: counter (bead,
 * run, step, 0); v0 NULL draws Maxwell-Boltzmann velocities at step0.
 * Shared memory bounds the chain (about 2900 beads).  Errors: RID_ERR_ARG,
 * RID_ERR_OOM, RID_ERR_CUDA, RID_ERR_NONFINITE.
 */
RID_API int rid_label_constrained(rid_system* sys, int32_t n_runs, const float* x0, const float* v0, int32_t n_cv,
                                  const int32_t* pairs, const double* d0, uint64_t step0, int64_t n_steps,
                                  int64_t n_equil, int32_t n_blocks, double* mf_out, double* se_out,
                                  double* std_out, float* x_out, float* v_out, int32_t mem, void* stream);

/*
 * Training the ensemble on mean-force labels (Sec. "Training phase":
 * numb_models, neurons, resnet, batch_size, init_lr, decay_steps, decay_rate;
 * Sec. "Training": the models are fitted to the labelled mean forces).
 *
 * Every member i has its own batches.  Its loss on a batch of B labels
 * (s_k, MF_k) is the mean over the batch and the C components of
 * (dA_i/ds_j(s_k) - MF_kj)^2, and its weights take one Adam step per batch
 * (beta1, beta2, adam_eps) with learning rate init_lr * decay_rate^(t /
 * decay_steps) at the trainer's t-th step (t = 0, 1, ...).  The weights use
 * the packed layout of rid_ensemble_desc.weights, so rid_trainer_weights can
 * feed rid_set_ensemble directly.  Arithmetic: FP32 with fixed summation
 * orders (a run is reproducible bit for bit); b_out does not enter the loss
 * and is never changed.
 *
 * Dropout (drop_out_rate of the training section; rate 0: off): inverted
 * dropout on the output of every hidden layer, h_l = q_l tanh(z_l) + r_l
 * h_{l-1}, in the forward pass and in the input gradient dA/ds of the loss
 * alike.  Unit j of layer l for batch row b of member m at step t is kept
 * (q = 1 / (1 - rate)) iff word j % 4 of Philox4x32-10 at counter
 * (j / 4 + ceil(H / 4) (l + L m), b, t, 4), key = dropout_seed, is at least
 * floor(rate 2^32), else dropped (q = 0).  rid_trainer_grad draws the masks
 * of the step the trainer would take next.
 *
 * All calls are synchronous on `stream`.  `mem` says where the array
 * arguments live (RID_MEM_HOST / RID_MEM_DEVICE).  Errors: RID_ERR_ARG (bad
 * sizes, a batch index outside [0, n_data): detected on the device, the step's
 * results are then not to be used), RID_ERR_STATE (no data), RID_ERR_OOM,
 * RID_ERR_CUDA.
 */
typedef struct {
    int32_t n_models;             /* M, 1..16                                   */
    int32_t n_cv;                 /* C (inputs D = 2C), 1..128                  */
    int32_t n_layers;             /* L, 1..8                                    */
    int32_t width;                /* H, 1..512                                  */
    int32_t resnet;               /* 0 / 1 (h_l = h_{l-1} + tanh(.) for l >= 2) */
    int32_t batch_size;           /* B, 1..65536 (128 in the paper)             */
    double init_lr;               /* 8e-4 in the paper                          */
    double decay_rate;            /* 0.96                                       */
    int32_t decay_steps;          /* 120                                        */
    double beta1, beta2, adam_eps;  /* Adam: 0.9, 0.999, 1e-8                   */
    double dropout_rate;          /* [0, 1): 0.1 in the paper, 0 = off          */
    uint64_t dropout_seed;        /* Philox key of the dropout masks            */
    const int32_t* cv_dist;       /* [C] host or NULL: 1 marks a distance CV,   */
                                  /* whose input pair is (s, 0) and dA/ds =     */
                                  /* dA/du_2j (read at creation, not kept)      */
} rid_train_desc;

typedef struct rid_trainer rid_trainer;

/* Create a trainer on the current device from host weights [M][P] (copied;
 * Adam moments start at zero, t = 0). */
RID_API int rid_trainer_create(const rid_train_desc* desc, const float* weights, rid_trainer** out);
RID_API int rid_trainer_destroy(rid_trainer* tr);
/* The label set: s [n][C] (radians) and mf [n][C], copied to the device. */
RID_API int rid_trainer_set_data(rid_trainer* tr, int32_t n, const float* s, const float* mf, int32_t mem,
                                 void* stream);
/* n_steps Adam steps; idx [n_steps][M][B] int32 are the sample indices of each
 * member's batch at each step; loss_out [n_steps][M] | NULL receives each
 * member's batch loss at the weights before its step. */
RID_API int rid_trainer_run(rid_trainer* tr, int32_t n_steps, const int32_t* idx, float* loss_out, int32_t mem,
                            void* stream);
/* The loss [M] and its gradient [M][P] at the current weights for one batch
 * idx [M][B], without changing the weights (either output may be NULL). */
RID_API int rid_trainer_grad(rid_trainer* tr, const int32_t* idx, float* loss_out, float* grad_out, int32_t mem,
                             void* stream);
/* Current weights [M][P] (NULL to skip) and the number of steps taken. */
RID_API int rid_trainer_weights(rid_trainer* tr, float* weights_out, int64_t* steps_done, int32_t mem,
                                void* stream);

/*
 * MCMC dimension reduction (Sec. "Dimension reduction phase": numb_walkers,
 * numb_steps, temperature, bins, proj_cv_index; Introduction, automatic PMF
 * calculation).  W walkers run Metropolis Monte Carlo on the torus of C
 * torsion CVs with the ensemble-mean free energy Abar(s) = (1/M) sum_i A_i(s)
 * at temperature kT:
 *   proposal  s' = wrap(s + step_size xi) per CV, xi = normal c % 3 of the
 *             Box-Muller triple of Philox counter (c / 3, walker, step, 2);
 *   accept    iff kT ln u + (Abar(s') - Abar(s)) < 0, u = (x + 1/2) 2^-32 with
 *             x = word 0 of counter (0, walker, step, 3) (key = seed);
 *   counting  from step n_burn on, each walker's current state after every
 *             step goes into hist1 [C][bins] (one histogram per CV) and hist2
 *             [bins][bins] (the pair proj_i, proj_j); bin =
 *             floor((s + pi) / (2 pi) * bins) clamped to [0, bins - 1];
 *   PMF       pmf = -kT ln(count / total) shifted to a zero minimum per
 *             histogram (+inf where a bin is empty), float64.
 * The ensemble is evaluated in FP32 (batched GEMMs).  s0 [W][C] holds the
 * starting CVs (radians); every output may be NULL.  Synchronous on `stream`;
 * device scratch is allocated for the call and released before it returns.
 * Errors: RID_ERR_ARG, RID_ERR_OOM, RID_ERR_CUDA.
 */
typedef struct {
    int32_t n_models;             /* M, 1..16                                   */
    int32_t n_cv;                 /* C (inputs D = 2C), 1..128                  */
    int32_t n_layers;             /* L, 1..8                                    */
    int32_t width;                /* H, 1..512                                  */
    int32_t resnet;               /* 0 / 1                                      */
    const float* weights;         /* [M][P] packed as rid_ensemble_desc.weights,
                                     host or device as `mem` says              */
    int32_t n_walkers;            /* W (2000 in the paper)                      */
    int64_t n_steps;              /* < 2^32                                     */
    int64_t n_burn;               /* steps before counting starts               */
    double kT;                    /* temperature in the energy unit of A        */
    double step_size;             /* proposal standard deviation (radians)      */
    uint64_t seed;                /* Philox key                                 */
    int32_t bins;                 /* per CV, 1..4096 (101 in the paper)         */
    int32_t proj_i, proj_j;       /* CV pair of the 2-D projection              */
    /* Path projection (the paper's "path" mode; off when path_n_nodes = 0):
     * path collective variables of nodes p_1..p_P over the CVs path_cv,
     * d_i = |s - p_i|^2 with wrapped differences,
     *   s_path = sum_i i e^{-lambda d_i} / sum_i e^{-lambda d_i},
     *   z_path = -(1/lambda) ln sum_i e^{-lambda d_i},
     * counted into hist_path [bins][bins] over [1, P] x [path_z_lo, path_z_hi]
     * (values clamped to the edge bins). */
    int32_t path_n_nodes;         /* P, 0 or 2..1024                            */
    int32_t path_n_cv;            /* CVs of the path, 1..C                      */
    const int32_t* path_cv;       /* [path_n_cv] host                           */
    const float* path_nodes;      /* [P][path_n_cv] host, radians               */
    double path_lambda;           /* > 0 (path_lm in the paper)                 */
    double path_z_lo, path_z_hi;  /* z range of hist_path                       */
    /* Distance CVs (the paper's cv_type "dis" with cv_lower_bound /
     * cv_upper_bound; NULL cv_dist: every CV a torsion).  A distance CV is
     * not periodic: its proposal s + step_size xi is not wrapped, a proposal
     * that takes any distance CV out of [cv_lo, cv_hi] is refused (the walk
     * samples exp(-Abar/kT) restricted to the box), its MLP input is (s, 0),
     * it is binned as floor((s - cv_lo) / (cv_hi - cv_lo) * bins) (clamped),
     * and path differences over it are plain. */
    const int32_t* cv_dist;       /* [C] host or NULL: 1 marks a distance CV    */
    const double* cv_lo;          /* [C] host: range of each distance CV        */
    const double* cv_hi;          /*   (entries of torsions are ignored)        */
} rid_mcmc_desc;

RID_API int rid_mcmc(const rid_mcmc_desc* desc, const float* s0, float* s_out, uint64_t* hist1, uint64_t* hist2,
                     double* pmf1, double* pmf2, uint64_t* hist_path, double* pmf_path, int64_t* n_accepted,
                     int32_t mem, void* stream);

/*
 * The same MCMC dimension reduction (proposal, rule, counting and PMF as
 * rid_mcmc) with the ensemble a system holds (rid_set_ensemble): the free
 * energy of each proposal is evaluated by the system's own ensemble kernels at
 * the precision the ensemble was set with (RID_PREC_FP32 / BF16 / FP8; the
 * tensor-core kernels for BF16 and FP8).  C is the system's CV count; s0
 * [W][C].  The system's resident walker buffers are reused (walkers loaded
 * with rid_walkers_load must be loaded again).  `path` (NULL, or n_nodes = 0:
 * off) adds the path projection of rid_mcmc_desc, with the same fields and
 * limits, counted into hist_path / pmf_path [bins][bins] (either may be NULL);
 * its arrays are host memory whatever `mem` says.  A system with distance CVs
 * (cv_atoms rows (a, b, -1, -1)) needs cv_lo / cv_hi [C] (host; the range of
 * each distance CV, torsion entries ignored), read as in rid_mcmc_desc; for a
 * torsion-only system they may be NULL.
 * Errors: RID_ERR_ARG, RID_ERR_STATE (no ensemble), RID_ERR_OOM, RID_ERR_CUDA.
 */
typedef struct {
    int32_t n_nodes;              /* P, 0 or 2..1024                            */
    int32_t n_cv;                 /* CVs of the path, 1..C                      */
    const int32_t* cv;            /* [n_cv] host                                */
    const float* nodes;           /* [P][n_cv] host, radians                    */
    double lambda;                /* > 0                                        */
    double z_lo, z_hi;            /* z range of hist_path                       */
} rid_mcmc_path;

RID_API int rid_mcmc_system(rid_system* sys, int32_t n_walkers, const float* s0, int64_t n_steps, int64_t n_burn,
                            double kT, double step_size, uint64_t seed, int32_t bins, int32_t proj_i, int32_t proj_j,
                            const double* cv_lo, const double* cv_hi, const rid_mcmc_path* path, float* s_out, uint64_t* hist1, uint64_t* hist2, double* pmf1,
                            double* pmf2, uint64_t* hist_path, double* pmf_path, int64_t* n_accepted, int32_t mem,
                            void* stream);

/*
 * Selection (Sec. "Selection phase": cluster_threshold, numb_cluster_lower,
 * numb_cluster_upper, max_selection; Sec. "Selection": explored CVs are
 * clustered and values with high model deviation are collected by the trust
 * levels; Sec. "CV selection": clustering weights and the angular mask).
 *   candidates  frames f with trust_lo <= eps[f] < trust_hi (compared in
 *               FP32), in frame order;
 *   distance    d^2 = sum_c w_c delta_c^2, delta = cv_a - cv_b wrapped onto
 *               [-pi, pi) for periodic CVs, FP32 with a fixed operation order;
 *   clustering  leader algorithm in candidate order: a candidate joins the
 *               first leader with d^2 <= t^2, else it becomes a leader (the
 *               representative of its cluster);
 *   adaptation  when adapt != 0 (the first iteration), t is searched from
 *               cluster_threshold until the cluster count falls in [lower,
 *               upper]: doubled / halved until bracketed, then geometric
 *               bisection, at most 63 more trials;
 *   output      selected[0 .. n_selected) = frame indices of the first
 *               max_selection leaders; n_clusters and the threshold used.
 * cv [n][C] and eps [n] are frames (e.g. rid_explore's traces flattened
 * walker-major); cv, eps and selected live where `mem` says; weights and
 * periodic are host arrays [C] (NULL: all 1 / all periodic); the scalar
 * outputs are host pointers (NULL to skip).  Synchronous on `stream`.
 * Errors: RID_ERR_ARG, RID_ERR_OOM, RID_ERR_CUDA.
 */
typedef struct {
    int32_t n_cv;                 /* C, 1..128                                  */
    const float* weights;         /* [C] host | NULL                            */
    const int32_t* periodic;      /* [C] host | NULL (angular_mask)             */
    double trust_lo, trust_hi;    /* candidate window on the model deviation    */
    double cluster_threshold;     /* t (initial guess when adapt != 0)          */
    int32_t numb_cluster_lower, numb_cluster_upper;
    int32_t adapt;                /* search t into [lower, upper]               */
    int32_t max_selection;        /* >= 0                                       */
} rid_select_desc;

RID_API int rid_select(const rid_select_desc* desc, int32_t n_frames, const float* cv, const float* eps,
                       int32_t* selected, int32_t* n_selected, int32_t* n_clusters, double* threshold_out,
                       int32_t mem, void* stream);

/*
 * One force evaluation at given positions (no integration), through the same
 * kernels as a step.  bias = RID_BIAS_*; s0/kappa [W][C] are read only for
 * RID_BIAS_RESTRAINT.
 *   f_out [W][N][3] float32   total force (force field + CV force)
 *   s_out [W][C], eps_out [W], abar_out [W], grad_out [M][W][C] (dA_i/ds),
 *   all float32 and optional (NULL).
 */
RID_API int rid_eval_forces(rid_system* sys, int32_t n_walkers, const float* x, int32_t bias,
                    const double* s0, const double* kappa, float* f_out, float* s_out,
                    float* eps_out, float* abar_out, float* grad_out, int32_t mem, void* stream);

/*
 * LJ pair inclusion of the force kernel, as a bit mask: bit (j & 31) of word
 * [w][i][j >> 5] is set iff the pair (i, j) interacts (|i-j| >= 3 and FP32
 * r^2 < rc^2, r^2 formed as in rid_system_desc).  mask_out [W][N][ceil(N/32)] uint32.
 */
RID_API int rid_pair_mask(rid_system* sys, int32_t n_walkers, const float* x, uint32_t* mask_out,
                  int32_t mem, void* stream);

/*
 * The integrator's random numbers for n given counters (bead, walker, step,
 * stream) under key `seed`: the Philox4x32-10 words (out_words [n][4] uint32)
 * and the three normals built from them (out_normals [n][3] float32).
 */
RID_API int rid_philox(int64_t n, const uint32_t* counters, uint64_t seed, uint32_t* out_words,
               float* out_normals, int32_t mem, void* stream);


/*
 * Resident walkers.  rid_explore is load + advance + read in one call; these
 * three let a caller keep the walker state on the device across calls (the
 * state lives in the system object; one walker set per system).
 *
 * rid_walkers_load: copy W walkers in (v0 NULL: Maxwell-Boltzmann draw at
 *   step0), set the global step counter to step0 and evaluate the forces at
 *   x0.  Synchronous.
 * rid_walkers_advance: n_steps biased (or, without an ensemble, unbiased)
 *   BAOAB steps from the resident state; traces as in rid_explore with
 *   T = n_steps / output_freq counted from the start of this call.  With
 *   mem = RID_MEM_DEVICE (or no trace outputs) the call only enqueues work on
 *   `stream` and returns; with host trace outputs it waits for completion.
 *   Non-finite results are reported by the next rid_walkers_read.
 * rid_walkers_read: wait for `stream`, copy positions / velocities out (either
 *   may be NULL), return the next global step index in *step_next (may be
 *   NULL), and report RID_ERR_NONFINITE if any walker went non-finite since
 *   the last load.
 */
RID_API int rid_walkers_load(rid_system* sys, int32_t n_walkers, const float* x0, const float* v0,
                             uint64_t step0, int32_t mem, void* stream);
RID_API int rid_walkers_advance(rid_system* sys, int64_t n_steps, float* cv_out, float* eps_out,
                                double* energy_out, int32_t mem, void* stream);
RID_API int rid_walkers_read(rid_system* sys, float* x_out, float* v_out, uint64_t* step_next,
                             int32_t mem, void* stream);

/*
 * Kernel timing for this system: while enabled, every kernel the system
 * launches is bracketed by CUDA events on its launch stream.  Enabling resets
 * the record.  rid_profile_read waits for the recorded events and returns, per
 * kernel name (in first-launch order, at most max_kernels), the summed
 * device time in milliseconds and the launch count; names_out receives
 * max_kernels slots of 48 bytes (NUL-terminated).  *n_kernels is the number
 * of distinct kernels recorded.  rid_launch_count returns the number of
 * kernels this system has launched since it was created.
 */
RID_API int rid_profile_enable(rid_system* sys, int32_t enable);
RID_API int rid_profile_read(rid_system* sys, int32_t max_kernels, char* names_out, double* total_ms,
                             int64_t* launches, int32_t* n_kernels);
RID_API int64_t rid_launch_count(rid_system* sys);

/*
 * Cluster size of the tensor-core ensemble kernel (BF16 / FP8 ensembles; no
 * counterpart in the paper, a tuning control).  The kernel splits every
 * GEMM's output columns over csize CTAs of a thread-block cluster (1: one CTA
 * per 128-walker tile and member; 2 or 4: the columns split over a cluster,
 * the next layer's operand exchanged through distributed shared memory).
 * csize = 0 (the default) lets the library time the force evaluation with
 * each eligible size at the first evaluation of every new walker count and
 * keep the fastest.  Every size gives the same results bit for bit.  BF16
 * ensembles evaluated for at most 16 walkers run a small-batch kernel instead
 * (the GEMMs transposed, each GEMM's 128-output tiles split over a cluster of
 * one CTA per tile, at most 4, or at most csize CTAs when csize is fixed; no
 * timing): its results agree with the other kernels within the BF16 bounds,
 * not bit for bit, depend only on the walker count and are the same bits for
 * every split.  While a
 * server runs an exploration job on the system (rid_submit), csize = 0 means 1
 * for the row kernels and nothing is timed: the request loop does not wait on
 * timing runs, and a size timed on an idle GPU is not the one for a shared
 * GPU.
 * Errors: RID_ERR_ARG (csize not 0, 1, 2 or 4); a size the ensemble's shape
 * does not allow (shared memory) fails with RID_ERR_ARG at the next
 * evaluation.
 */
RID_API int rid_set_mlp_cluster(rid_system* sys, int32_t csize);

/*
 * Cluster size of the tensor-core ensemble kernel's last launch (as tuned or
 * as fixed by rid_set_mlp_cluster), written to the host int csize; 0 before
 * any BF16 / FP8 ensemble evaluation and for FP32 ensembles.
 * Errors: RID_ERR_ARG (NULL argument).
 */
RID_API int rid_get_mlp_cluster(rid_system* sys, int32_t* csize);

/*
 * CTA size of the force-field kernel (threads per walker CTA: beads per pass
 * and CTAs per SM; a tuning control, no counterpart in the paper).  threads =
 * 0 (the default) lets the library time the kernel with every multiple of 32
 * from 64 up to its default size (the chain's bead count rounded up to 32, at
 * most 224) at the first force evaluation of every new walker count and keep
 * the fastest (the default, untimed, while a server runs a job on the
 * system).  Forces are the same bits with every size; force-field energy
 * evaluations always use the default size.  With fewer walkers than two per
 * SM (no setting: from the shape alone) each walker's passes over its chain
 * are split over up to 8 CTAs, and the integrator kernel runs each walker as a
 * thread-block cluster of up to 8 CTAs over its bead batches (not for energy
 * evaluations, nor while a server runs a job on the system); results are the
 * same bits either way.
 * Errors: RID_ERR_ARG (threads not 0 or a multiple of 32 in [32, default]).
 */
RID_API int rid_set_ff_threads(rid_system* sys, int32_t threads);

/*
 * The force-field CTA size in use (host int written): the fixed one, the
 * tuned one for the last walker count, or the default before any evaluation.
 * Errors: RID_ERR_ARG (NULL argument).
 */
RID_API int rid_get_ff_threads(rid_system* sys, int32_t* threads);

/*
 * Fused exploration steps (no counterpart in the paper, a tuning control): on
 * = 1 (the default) runs every step of an exploration call (rid_explore,
 * rid_walkers_advance) in one persistent launch, one CTA per walker holding
 * its chain, CVs and the whole ensemble in shared memory, when the ensemble is
 * FP32 and non-residual with at most 8 members, the chain has at most 128
 * beads, the CVs number at most 32, the state fits the CTA's shared memory,
 * the walkers fit one wave of CTAs, and no energy trace is asked for;
 * otherwise, and with on = 0, the steps run as per-step kernels.
 * The switch also sends rid_label of chains below 768 beads through the
 * persistent label kernel (every step of every run in one launch, one CTA per
 * run).  Each step is the per-step kernels' arithmetic in the same order, so
 * the results are the same bits either way; a fused call ends with its last
 * step closed.
 * Errors: RID_ERR_ARG (sys NULL, or on not 0 or 1).
 */
RID_API int rid_set_fused_steps(rid_system* sys, int32_t on);

/*
 * Server: device memory of a fixed HBM budget, from which batched label runs
 * (rid_label_batch) and the request loop (rid_submit / rid_poll) take their
 * device memory.  Memory is allocated in segments, on demand, up to the
 * budget, on the device current at rid_server_create; every later call must
 * be made with that device current.  rid_submit and rid_poll may be called
 * from any thread; rid_label_batch and rid_server_destroy from one thread at
 * a time.  rid_server_destroy waits for every submitted job to finish.
 * Exploration jobs run on up to 16 streams of their own.  The CUDA runtime
 * maps a process's streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware work
 * queues (8 unless the variable is set, at most 32) and streams sharing a
 * queue wait on one another's launches, so a process that serves should set
 * it to 32 before its first CUDA call (the Python binding does so at import
 * unless it is already set).
 * Errors: RID_ERR_ARG (budget below 1 MiB), RID_ERR_OOM (the budget cannot be
 * allocated), RID_ERR_CUDA.
 */
typedef struct rid_server rid_server;
RID_API int rid_server_create(uint64_t hbm_budget_bytes, rid_server** out);
RID_API int rid_server_destroy(rid_server* srv);   /* NULL is accepted */

/* One restrained labeling job of a batch.  Every field means what the
 * argument of the same name means for rid_label; `sys` is the job's chain,
 * force field, CVs and integrator (any number of jobs may share a system). */
typedef struct {
    rid_system* sys;
    int32_t n_runs;             /* R >= 1                                        */
    int32_t n_blocks;           /* 2..256, n_steps - n_equil >= n_blocks         */
    const float* x0;            /* [R][N][3]                                      */
    const float* v0;            /* [R][N][3] | NULL (Maxwell-Boltzmann at step0)  */
    const double* s0;           /* [R][C]                                         */
    const double* kappa;        /* [R][C]                                         */
    uint64_t step0;
    int64_t n_steps, n_equil;
    double* mf_out;             /* [R][C]                                         */
    double* se_out;             /* [R][C]                                         */
    double* std_out;            /* [R][C]                                         */
    float* x_out;               /* [R][N][3] | NULL                               */
    float* v_out;               /* [R][N][3] | NULL                               */
} rid_label_job;

/*
 * Batched restrained labeling (Sec. "Labeling phase", restrained method):
 * every run of every job in ONE persistent kernel launch that keeps each
 * chain resident in shared memory for all of its steps.  Jobs may differ in
 * chain length, CV count, restraints and step counts.  Each job's outputs are
 * bit-identical to rid_label on the same inputs.
 *   threads     CTA size of the persistent kernel: 128, 256 or 512, or 0 to
 *               pick it by timing the batch itself for a few steps (the
 *               choice is cached per batch shape on the server)
 *   status_out  [n_jobs] | NULL: per job RID_OK or RID_ERR_NONFINITE
 * `mem` applies to every array of every job.  Synchronous.  The jobs' device
 * memory comes from the server pool and is released before the call returns.
 * Errors: RID_ERR_ARG (a job violates a rid_label limit, or its chain needs
 * more than 220 KB of shared memory: about 4000 beads), RID_ERR_OOM (the batch
 * does not fit the server's budget), RID_ERR_STATE (wrong device),
 * RID_ERR_CUDA, RID_ERR_NONFINITE (some job went non-finite; outputs written).
 */
RID_API int rid_label_batch(rid_server* srv, const rid_label_job* jobs, int32_t n_jobs, int32_t threads,
                            int32_t* status_out, int32_t mem, void* stream);

/*
 * Request loop (continuous batching).  rid_submit queues a labeling or an
 * exploration job and returns at once; a worker thread of the server admits
 * queued jobs in arrival order as soon as their device memory fits the
 * budget (a job that does not fit holds back the jobs behind it; an
 * exploration job waiting for one of the 16 exploration streams or for its
 * system does not), and runs every admitted job concurrently:
 *   - label jobs advance together, in ticks of the persistent kernel
 *     (rid_label_batch's kernel); each tick gives every active job a number
 *     of steps sized to its chain length, and jobs that arrive meanwhile join
 *     the next tick;
 *   - exploration jobs run on their own stream as captured CUDA graphs of a
 *     chunk of steps, replayed until the job is done (one graph per job).
 * A job's results are the same bits as rid_label / rid_explore on the same
 * inputs, alone or in any mix.
 * Memory: label jobs take their arrays from the server pool; an exploration
 * job's system holds its own device state, which the server counts against
 * the same budget (the bytes of its walker state and ensemble scratch) while
 * the job runs.
 */
enum { RID_JOB_LABEL = 1, RID_JOB_EXPLORE = 2 };

typedef struct {
    int32_t kind;             /* RID_JOB_LABEL or RID_JOB_EXPLORE                         */
    int32_t n_walkers;        /* label runs R, or exploration walkers W                    */
    rid_system* sys;          /* the job's chain; for exploration also its ensemble.  An
                                 exploration job uses the system's resident walker state:
                                 exploration jobs on one system run one after another,
                                 and the caller must not use the system until rid_poll
                                 reports the job final                                  */
    const float* x0;          /* host [W][N][3], copied by rid_submit                      */
    const float* v0;          /* host [W][N][3] | NULL (Maxwell-Boltzmann at step0)        */
    uint64_t step0;
    int64_t n_steps;
    /* labeling (see rid_label) */
    const double* s0;         /* host [R][C], copied                                       */
    const double* kappa;      /* host [R][C], copied                                       */
    int64_t n_equil;
    int32_t n_blocks;
    double* mf_out;           /* host [R][C]                                              */
    double* se_out;
    double* std_out;
    /* exploration (see rid_explore) */
    float* cv_out;            /* host [W][T][C] | NULL                                     */
    float* eps_out;           /* host [W][T] | NULL                                        */
    /* both */
    float* x_out;             /* host [W][N][3] | NULL                                     */
    float* v_out;             /* host [W][N][3] | NULL                                     */
} rid_request;

/* Times in milliseconds since the server was created. */
typedef struct {
    int32_t status;           /* RID_NOT_READY or the job's final status                  */
    int32_t kind;
    double t_submit_ms;
    double t_start_ms;        /* admitted (device memory granted), -1 while queued         */
    double t_end_ms;          /* results written, -1 while running                         */
} rid_job_info;

/* Queue a job.  Output arrays must stay valid until rid_poll reports the job
 * final.  Errors (nothing queued): RID_ERR_ARG (a rid_label / rid_explore
 * limit, host arrays only), RID_ERR_STATE (system on another device),
 * RID_ERR_OOM (the job alone exceeds the budget). */
RID_API int rid_submit(rid_server* srv, const rid_request* req, uint64_t* job_id);
/* Non-blocking: RID_NOT_READY while the job is queued or running, else its
 * final status (RID_OK, RID_ERR_NONFINITE with outputs written, RID_ERR_CUDA,
 * ...), after which the id is forgotten.  info (may be NULL) is filled in
 * either case.  Unknown id: RID_ERR_ARG. */
RID_API int rid_poll(rid_server* srv, uint64_t job_id, rid_job_info* info);
/* Withdraw a job that is still queued (not yet admitted; it holds no device
 * memory and no device work of it has been issued): the job is dropped, its
 * output arrays are not written, and rid_poll then reports RID_ERR_CANCELLED
 * (t_start_ms stays -1).  A host-side operation: no device call.  Errors:
 * RID_ERR_ARG (srv NULL, or an unknown or already polled id), RID_ERR_STATE
 * (the job is running or final: it runs to its end and rid_poll reports its
 * own status). */
RID_API int rid_cancel(rid_server* srv, uint64_t job_id);
/* Jobs queued and running, and device bytes granted to running jobs. */
RID_API int rid_server_load(rid_server* srv, int32_t* queued, int32_t* running, uint64_t* bytes_in_use);

/*
 * Ensemble member gradients with no device allocation.  The paper has no
 * counterpart: this is a library facility for callers that cannot allocate
 * device memory.  Two kinds of caller need it: a host framework that hands
 * out all device memory from its own pool (a cudaMalloc behind its back is
 * memory its accounting does not see, and fails once the pool has reserved
 * the device), and an embedding that forbids allocation after start-up
 * (cudaMalloc can synchronise the device and take unbounded time, which a
 * latency-bound or certified code path cannot allow).
 *
 * For P points s [P][C] (device, float32, radians) and the packed ensemble
 * `weights` [M][Pw] (device, float32, the layout of rid_ensemble_desc.weights,
 * D = 2C inputs (cos s_j, sin s_j)) it writes
 *   grad_out  [M][P][C] float32 (device)        dA_i/ds at every point
 *   value_out [M][P]    float32 (device) | NULL A_i at every point
 * with the arithmetic of the RID_PREC_FP32 ensemble kernel.  All arrays belong
 * to the caller; the call enqueues one kernel on `stream` and returns.
 *
 * Scratch: the hidden activations kept for the reverse pass live in one
 * static 8 MiB device array per device, so M * ceil(P/32) * 32 * L * H must
 * not exceed 2^21 floats (e.g. P = 1024, M = 4, L = 4, H = 128); larger
 * requests return RID_ERR_ARG without launching.  The array keeps the last
 * call's contents; nothing in it needs to start at zero (every entry read is
 * written earlier by the same kernel).  Calls that overlap in time on one
 * device (two streams, or two threads) share the array and race: serialise
 * them.  The first call on a device (with that device current) looks up the
 * array's address with cudaGetSymbolAddress and sets the kernel's shared
 * memory limit; make that first call before any stream capture.
 * Errors: RID_ERR_ARG (NULL array, sizes outside the limits of
 * rid_ensemble_desc, scratch too small), RID_ERR_CUDA.
 */
RID_API int rid_ensemble_grad_noalloc(int32_t n_points, int32_t n_cv, const float* s, int32_t n_models,
                                      int32_t n_layers, int32_t width, int32_t resnet, const float* weights,
                                      float* grad_out, float* value_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RID_H */
