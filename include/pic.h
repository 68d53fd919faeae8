/*
 * pic.h - C ABI of the GB300 electrostatic PIC library (Landau damping).
 *
 * The library advances the electrostatic Vlasov-Poisson system of the paper
 * (Sec. 2, Eqs. 1-4) with the particle-in-cell loop of Fig. 1:
 * scatter -> solve -> gather -> push, on one GPU. The solve is a matrix-free
 * preconditioned conjugate gradient on the periodic 7-point finite-difference
 * Laplacian (Sec. 3.2; Jacobi, a learned CNN, a multigrid V-cycle or the
 * paper's SSOR as the preconditioner), or the FFT pseudo-spectral solve of
 * Sec. 3.1. All calls are plain C: device buffers are passed as raw
 * pointers, sizes as integers, and no C++ exception crosses the boundary.
 *
 * Conventions (Sec. 2 and Sec. 2.1):
 *   - plasma units: electrons with q/m = -1, eps0 = 1, mean density 1, so the
 *     neutralising ion background is +1 and Poisson's equation reads
 *     -Delta phi = rho (Eq. 2), E = -grad phi;
 *   - periodic cube [0, L)^3, L = 2 pi / k, N^3 nodes x_i = i h, h = L / N;
 *   - grid arrays are N^3 contiguous values, x fastest: i + N (j + N k);
 *   - particles live in the context as 64-byte records (the cell and a 64-bit
 *     fixed-point offset inside it per coordinate, double-float velocities);
 *     pic_get_particles returns them in FP64, structure of arrays.
 *
 * Streams: every call enqueues its work on the context's CUDA stream
 * (given to pic_create) and returns without synchronising, except those that
 * return host values (pic_field_energy, pic_get_particles to host memory,
 * poisson_solve*, which read convergence status), which synchronise the stream.
 *
 * Errors: every int-returning call returns PIC_OK (0) or a negative code;
 * pic_strerror() names it. After PIC_ECUDA the context should be destroyed.
 * The library never traps or asserts on the device: device-side failures
 * (non-finite values, breakdown, exhausted waits) are reported through the
 * return codes below.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_EINVAL -1     /* bad argument (null pointer, unsupported size, ...) */
#define PIC_ENOMEM -2     /* device or pinned allocation failed */
#define PIC_ECUDA -3      /* a CUDA runtime call failed */
#define PIC_ENOCONV -4    /* solver hit maxit; phi holds the last iterate */
#define PIC_EBREAKDOWN -5 /* solver breakdown: p.Ap <= 0 or a non-finite value */
#define PIC_ETIMEOUT -6   /* a bounded device-side wait expired */
#define PIC_ESTATE -7     /* call out of order (e.g. deposit before init) */

typedef struct pic_ctx pic_ctx;

/* Problem description (Sec. 2.1: k = 0.5, alpha = 0.05; Sec. 4.1: 8 ppc). */
typedef struct {
  int N;         /* nodes per dimension; 8 <= N <= 1024, N % 8 == 0 */
  int ppc;       /* particles per cell, Np = ppc * N^3 < 2^32; 0 = solver-only context */
  double alpha;  /* density perturbation amplitude, |alpha| < 1 (< 1/3 with init_mode 1) */
  double k;      /* perturbation wavenumber; L = 2 pi / k */
  double vth;    /* thermal velocity of the Maxwellian (0 selects 1, the paper's units) */
  int init_mode; /* 0: the paper's density prod_d (1 + alpha cos k x_d);
                    1: the sum form 1 + alpha sum_d cos k x_d */
} pic_params;

/* Solver precision. FP64 = Jacobi-PCG entirely in FP64 (the reference solve).
 * MIXED = FP32 stencil and vectors, FP64 reductions, FP64 solution and
 * reliable-update residual recomputation in FP64. */
enum { PIC_PREC_FP64 = 0, PIC_PREC_MIXED = 1 };
/* Preconditioner: JACOBI (Sec. 3.2); the learned CNN inside flexible CG
 * (requires PIC_PREC_MIXED and weights set by pic_cnn_set_weights); a
 * geometric multigrid V-cycle inside flexible CG (beyond the paper, whose
 * conclusion, Sec. 5, sets PCG beside the multigrid solvers of a cited
 * comparison; requires PIC_PREC_MIXED): MG smooths every level with
 * damped Jacobi, MG_CNN smooths the finest level with the learned network
 * (requires weights). See pic_mg_apply for the cycle. SSOR is the paper's
 * PCG configuration (Sec. 4.1, red-black ordering, 4 inner and 2 outer
 * iterations, damping pi/2; requires PIC_PREC_MIXED); see pic_ssor_apply. */
enum { PIC_PC_JACOBI = 0, PIC_PC_CNN = 1, PIC_PC_MG = 2, PIC_PC_MG_CNN = 3, PIC_PC_SSOR = 4 };

typedef struct {
  int precision;         /* PIC_PREC_* */
  int precond;           /* PIC_PC_* */
  double reliable_delta; /* MIXED: recompute the FP64 residual when the FP32 residual
                            norm fell by this factor since the last recomputation
                            (1e-4 <= reliable_delta < 1, else PIC_EINVAL: below
                            1e-4 the FP32 recursion runs out of precision first);
                            0 selects the default: 0.1 with Jacobi, 0.03 with
                            the learned preconditioner, 0.001 with the V-cycle */
  int check_every;       /* iterations between host reads of the convergence flag;
                            0 = default (1 with the V-cycle, 32 up to 64^3, else 8) */
  int refine_max;        /* MIXED: at most this many FP64 residual recomputations (the
                            refinement steps of the inner FP32 solve, each after the FP32
                            residual fell by reliable_delta, the inner tolerance); when
                            reached unconverged the solve stops with PIC_ENOCONV; 0 = no cap */
} pic_solve_opts;

typedef struct {
  int iters;            /* CG iterations performed */
  int reliable_updates; /* MIXED: FP64 residual recomputations */
  int fallbacks;        /* CNN: iterations that used the Jacobi direction */
  int converged;        /* 1 if ||b - A phi|| <= tol ||b|| */
  double rel_res;       /* final ||r|| / ||b|| (FP64 recursive residual for FP64,
                           true FP64 residual b - A phi for MIXED) */
  double bnorm;         /* ||b||_2 of the mean-projected right-hand side */
  double t_ms;          /* device time of the solve (CUDA events) */
} pic_solve_info;

/* Create a context on the current CUDA device. `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream); the caller keeps it alive for
 * the context's lifetime. The context owns its particles and workspace. */
int pic_create(pic_ctx **out, void *cuda_stream);
void pic_destroy(pic_ctx *c);
const char *pic_strerror(int code);
/* Name of the CUDA runtime error behind the calling thread's most recent
 * PIC_ECUDA (e.g. "cudaErrorMemoryAllocation"), or "no CUDA error". */
const char *pic_cuda_error(void);

/* S0 (Sec. 2.1): allocate and sample the Landau initial condition on the
 * device. Particle p draws from Philox4x32-10 (Salmon et al., SC'11) with
 * counters (p_lo, p_hi, j, 0) and key (seed_lo, seed_hi). init_mode 0:
 * positions by per-dimension inverse CDF of (1 + alpha cos k x)/L (calls
 * j = 0, 1); init_mode 1: positions from the sum density by rejection from
 * the uniform one (trial t uses calls 4 + 2t and 5 + 2t, at most 32 trials).
 * Velocities: vth times Box-Muller normals (calls 2, 3), synchronous with the
 * positions. With ppc == 0 only the grid geometry is set (solver-only
 * context). PIC_EINVAL for parameters out of range. */
int pic_init(pic_ctx *c, const pic_params *p, uint64_t seed);

/* S1 + S2 (Fig. 1 "scatter", Eq. 2): sort particles by cell, then write
 * rho = 1 + sum_p q_p W_CIC(x_i - x_p) / h^3, q_p = -L^3/Np, into `rho`
 * (device FP64 [N^3], caller-owned; fully overwritten). */
int pic_deposit(pic_ctx *c, double *rho);

/* S3 + S4 (Sec. 3.2, 4.1): solve A phi = rho - mean(rho), A = -Delta_h the
 * periodic 7-point operator, by Jacobi-PCG in FP64 until
 * ||r||_2 <= tol ||b||_2 or maxit iterations. `rho` (device FP64 [N^3]) is
 * read only. `phi` (device FP64 [N^3]) is in/out: on entry the warm start,
 * on return the solution with mean zero. Returns PIC_OK, PIC_ENOCONV (phi =
 * last iterate) or PIC_EBREAKDOWN. A zero right-hand side gives phi = 0. */
int poisson_solve(pic_ctx *c, const double *rho, double *phi, double tol, int maxit);

/* As poisson_solve with solver options (NULL = FP64 Jacobi) and an optional
 * info record (NULL = not filled). */
int poisson_solve_ex(pic_ctx *c, const double *rho, double *phi, double tol, int maxit,
                     const pic_solve_opts *opts, pic_solve_info *info);

/* S5 + S6 (Eq. 2, Eqs. 3-4; Fig. 1 "gather", "push"): E = -grad phi by
 * central differences, CIC-gathered to the particles, then one leapfrog step:
 * v += (q/m) kick E(x), x = wrap(x + dt v), where kick = dt/2 on the first
 * push after pic_init / pic_sync_velocity and dt otherwise (kick-drift-kick
 * with the two half-kicks at each step boundary merged). `phi` is device
 * FP64 [N^3]. PIC_EINVAL for a non-finite dt. A particle whose kick is not
 * finite (a non-finite phi near it) is left unchanged and the context records
 * the fault: its next synchronising call returns PIC_EBREAKDOWN, and so do
 * the later ones (destroy the context). */
int pic_gather_push(pic_ctx *c, const double *phi, double dt);

/* Closing half-kick v += (q/m) (dt/2) E(x): makes velocities synchronous
 * with positions again (for diagnostics); the next push starts with dt/2. */
int pic_sync_velocity(pic_ctx *c, const double *phi, double dt);

/* S7 (Fig. 2 diagnostic): out_w[d] = h^3 sum_i E_{d,i}^2, E = -grad phi by
 * central differences, d = x, y, z. `out_w` is host memory; synchronises. */
int pic_field_energy(pic_ctx *c, const double *phi, double out_w[3]);

/* The red-black SSOR preconditioner by itself: z = M r on the scaled system
 * (h^2 A) z = r, r and z device FP32 [N^3] (z is overwritten; r is not). From
 * z = 0, two outer iterations of four forward SOR sweeps (red nodes, then
 * black; red when i + j + k is even) and four backward sweeps (black, then
 * red), damping pi/2 (Sec. 4.1); FP32. Enqueued on the context stream. */
int pic_ssor_apply(pic_ctx *c, const float *r, float *z);

/* The FFT pseudo-spectral periodic solve (Sec. 3.1), the paper's other
 * solver: phi = F^-1(rho_hat / k^2) and, when E is not NULL,
 * E_d = F^-1(-i k_d rho_hat / k^2), k = 2 pi m / L (3-D FP64 transforms by
 * cuFFT). The k = 0 mode is zero (rho's mean is removed; phi has mean zero);
 * for the derivative along d its Nyquist mode m_d = N/2 is zero. rho, phi:
 * device FP64 [N^3], x fastest (rho is not modified); E: device FP64
 * [3 N^3] (E_x, E_y, E_z) or NULL. The context keeps the transform plans and
 * two complex buffers of N^2 (N/2 + 1) values. Returns PIC_ECUDA if cuFFT
 * fails (including out of memory for its plans). */
int pic_fft_solve(pic_ctx *c, const double *rho, double *phi, double *E);

/* S6 with a given node field instead of -grad phi (the FFT scheme's spectral
 * field): E device FP64 [3 N^3] (E_x, E_y, E_z). Same leapfrog as
 * pic_gather_push. */
int pic_gather_push_field(pic_ctx *c, const double *E, double dt);

/* pic_sync_velocity with a given node field E (device FP64 [3 N^3]). */
int pic_sync_velocity_field(pic_ctx *c, const double *E, double dt);

/* S7 from a given node field: out_w[d] = h^3 sum_i E_{d,i}^2 (host memory;
 * synchronises). */
int pic_field_energy_E(pic_ctx *c, const double *E, double out_w[3]);

/* The particle-in-Fourier field (Sec. 3.4, Appendix A), the paper's third
 * scheme: the charges go to the Fourier modes K_N (N = the grid size, modes
 * -N/2..N/2-1) by a type-1 NUFFT, E_hat = -i k rho_hat / (|k|^2 L^3) over
 * the symmetric modes |m_d| <= N/2 - 1 (k != 0), and the field is evaluated
 * at the particles by a type-2 NUFFT (exponential-of-semicircle window of
 * w = ceil(-log10 tol) + 1 points, 4 <= w <= 16, on a 2x oversampled grid,
 * FP64 arithmetic and cuFFT; the error is about tol relative to the field's
 * maximum, down to ~1e-12). The particles are first sorted by cell (as by
 * pic_deposit). E: device FP64 [3 Np] (E_x, E_y, E_z) in the ORIGINAL
 * particle order (index p of pic_init). The oversampled grids take about
 * 320 bytes per Fourier mode (kept between calls with the same N and w).
 * PIC_EINVAL for tol <= 0 or NaN, PIC_ESTATE without particles. */
int pic_pif_field(pic_ctx *c, double tol, double *E);

/* One leapfrog step of the particle-in-Fourier scheme: the PIF field at the
 * particles (no grid deposit or solve), then the kick and drift of
 * pic_gather_push (the first step after pic_init kicks by dt/2). PIC_EINVAL
 * for tol <= 0 or NaN or a non-finite dt, PIC_ESTATE without particles. */
int pic_pif_push(pic_ctx *c, double tol, double dt);

/* Self-test of the library's bounded device-side waits (the mbarrier waits of
 * the streaming solver kernels and of the tensor-core preconditioner, which
 * give up after about two seconds instead of hanging): one warp waits on an
 * mbarrier of one expected arrival, with a wall-time budget of budget_ns
 * (1 <= budget_ns <= 2e9). With producer = 1 a lane arrives and the call
 * returns PIC_OK; with producer = 0 nothing arrives (no copy is issued), the
 * wait runs out and the call returns PIC_ETIMEOUT; the context keeps the
 * timeout recorded, as after any expired wait: its later synchronising
 * calls return PIC_ETIMEOUT, so destroy it. Synchronises. PIC_EINVAL for a
 * budget or producer out of range. */
int pic_selftest_bounded_wait(pic_ctx *c, uint64_t budget_ns, int producer);

/* Copy particles out as 6 SoA blocks of Np doubles (x, y, z, vx, vy, vz) in
 * the ORIGINAL particle order (index p of pic_init), to device memory
 * (on_device = 1) or host memory (0; pageable or pinned; converted and copied
 * in chunks of 2^24 particles through a context-owned 805 MB device staging
 * buffer; synchronises). `half_step` (may be NULL) receives 1 when
 * velocities lag positions by dt/2. */
int pic_get_particles(pic_ctx *c, double *out, int on_device, int *half_step);

/* Replace the particle state (the phase-space sample f of Sec. 2 that the
 * loop of Fig. 1 advances) by caller data, the inverse of pic_get_particles:
 * `in` holds 6 SoA blocks of Np doubles (x, y, z, vx, vy, vz), Np =
 * pic_num_particles; element p becomes particle p. Positions are wrapped
 * into [0, L) (any finite value is accepted); velocities are stored as
 * double-float pairs (~48-bit significand), positions as the cell and a
 * 64-bit fixed-point offset. `half_step` = 1 states that the velocities lag
 * the positions by dt/2 (the next push kicks by dt), 0 that they are
 * synchronous (the next push kicks by dt/2). From device memory (on_device =
 * 1, 8-byte aligned, read only) or host memory (0; pageable or pinned; copied
 * in chunks of 2^24 particles through the staging buffer of
 * pic_get_particles). Synchronises. Returns PIC_EINVAL for a null pointer, a
 * half_step other than 0/1, or a non-finite value in `in` (the state is then
 * replaced with those particles at the origin at rest: set it again),
 * PIC_ESTATE for a context without particles. */
int pic_set_particles(pic_ctx *c, const double *in, int on_device, int half_step);

/* Number of particles of the context (0 for a solver-only context). */
int64_t pic_num_particles(const pic_ctx *c);

/* Operator application y = A x (A = -Delta_h, periodic 7-point, Sec. 3.2),
 * FP64 device [N^3] arrays. */
int pic_apply_laplacian(pic_ctx *c, const double *x, double *y);

/* Residual of the solve's system (Sec. 3.2): r = (rho - mean rho) - A (phi -
 * mean phi), FP64 device [N^3] arrays (used to build training snapshots). */
int pic_residual(pic_ctx *c, const double *rho, const double *phi, double *r);

/* ------------------------------------------------------------------------
 * Learned preconditioner (used with PIC_PC_CNN inside flexible CG). The paper
 * lists Jacobi, Richardson, Gauss-Seidel and SSOR preconditioners for its PCG
 * solver (Sec. 3.2); this one is a 4-layer 3x3x3 conv3d network
 * 1 -> 16 -> 16 -> 16 -> 1 channels, no biases, identity activations,
 * periodic padding, whose layers 3 and 4 are the adjoints of layers 2 and 1
 * (channels transposed, taps flipped): N = G^T G is symmetric positive
 * semi-definite for any weights (a learned factorised sparse approximate
 * inverse). BF16 weights and activations, FP32 accumulation on the tensor
 * cores. As a preconditioner it maps a residual r to z = s N(r / s), s = RMS(r).
 *
 * Weights (14 688 FP32 values) are the four layers concatenated, each in
 * the order w[out][in][tz][ty][tx] with tap offset (tz-1, ty-1, tx-1):
 * y[o, p] = sum_{c,t} w[o, c, t] x[c, p + t - 1].
 * Training arrays are B cubic crops of D^3 cells (D % 16 == 0), FP32, x fastest.
 * ------------------------------------------------------------------------ */
#define PIC_CNN_WEIGHTS 14688

/* Set the FP32 master weights from host memory (resets Adam); layers 3 and 4
 * are replaced by the adjoints of layers 2 and 1. Synchronises. */
int pic_cnn_set_weights(pic_ctx *c, const float *w_host);
/* Copy the FP32 master weights / accumulated gradients to host memory. */
int pic_cnn_get_weights(pic_ctx *c, float *w_host);
int pic_cnn_get_grads(pic_ctx *c, float *g_host);

/* Preconditioner on the context grid: z = N r for device FP32 [N^3] r, z
 * (periodic). N is linear, so it equals one 9^3 convolution with the composed
 * kernel K (rebuilt from the master weights at every weight update). How it
 * is evaluated on grids with N % 32 == 0 is set by pic_cnn_set_apply; other
 * grids (N % 16 == 0) always run the four BF16 tensor-core convs. */
int pic_cnn_apply(pic_ctx *c, const float *r, float *z);

/* One multigrid V-cycle z = V(r) on the context grid (device FP32 [N^3],
 * periodic), for the scaled system (6 I - adj) z = r, i.e. r = h^2 times the
 * physical residual. Levels N, N/2, ... while even and above 4 (the coarsest:
 * 40 damped Jacobi sweeps); full-weighting restriction (coarse right-hand
 * side 4 R r), trilinear prolongation (R = P^T / 8); two damped-Jacobi
 * sweeps (omega = 6/7) before and after the coarse-grid correction on every
 * level, or, with learned != 0, one application of the network before and
 * after on the finest level (requires weights). Levels of at most 16^3 run
 * in one thread block. */
int pic_mg_apply(pic_ctx *c, const float *r, float *z, int learned);

/* Evaluation of the preconditioner (pic_cnn_apply and the solver's
 * preconditioner step) on grids with N % 32 == 0:
 *   PIC_CNN_APPLY_TC     composed kernel on the tensor cores (N % 128 == 0):
 *                        x-direction Toeplitz products over 16 outputs and
 *                        32 inputs (two K = 16 MMA steps per (plane, dy)), r
 *                        and K rounded to BF16, FP32 accumulation (default);
 *                        on grids that are not a multiple of 128 this mode
 *                        runs PIC_CNN_APPLY_FP32;
 *   PIC_CNN_APPLY_FP32   composed kernel on the CUDA cores, FP32 throughout;
 *   PIC_CNN_APPLY_LAYERS the four BF16 tensor-core convs of the network;
 *   PIC_CNN_APPLY_TC_FUSED as PIC_CNN_APPLY_TC, and flexible CG runs its
 *                        residual/solution update and the direction's dot
 *                        products inside the preconditioner kernel (one pass
 *                        instead of three; N % 128 == 0, else as TC);
 *   PIC_CNN_APPLY_TC8    the same products over 8 outputs and 16 inputs (one
 *                        K = 16 step, 9 of 16 weights nonzero against 9 of
 *                        32), kept for comparison: it issues twice the MMAs
 *                        per output and runs slower on GB300 (one thread's
 *                        MMA issue, not the tensor work, bounds both forms);
 *                        the same sums in another order, so its result
 *                        differs from TC by FP32 rounding only.
 * Returns PIC_EINVAL for another mode. */
enum {
  PIC_CNN_APPLY_TC = 0,
  PIC_CNN_APPLY_FP32 = 1,
  PIC_CNN_APPLY_LAYERS = 2,
  PIC_CNN_APPLY_TC_FUSED = 3,
  PIC_CNN_APPLY_TC8 = 4
};
int pic_cnn_set_apply(pic_ctx *c, int mode);

/* Forward pass over B crops: y = N(x) (device FP32 [B][D^3] each); keeps the
 * activations for pic_cnn_backward. */
int pic_cnn_forward(pic_ctx *c, const float *x, float *y, int B, int D);
/* Backward pass of the last forward: adds d(sum gy * y)/dw of the tied
 * network to the gradients (layers 1 and 2 receive their own gradient plus
 * the adjoint of layer 4's and 3's; layers 3 and 4 hold the adjoints of
 * those sums). Data gradients run as adjoint convolutions on the tensor
 * cores, weight gradients on the CUDA cores in FP32. */
int pic_cnn_backward(pic_ctx *c, const float *gy, int B, int D);
/* One Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) on the
 * accumulated gradients, which are then zeroed. */
int pic_cnn_adam(pic_ctx *c, double lr);

/* Training batch from CG snapshots on the context grid: B periodic crops of
 * D^3 cells (D % 16 == 0) at host origins (3 ints per crop, x y z) of the
 * residual field r and of the error e = a - b (a = converged solution, b =
 * iterate), all device FP64 [N^3]. Writes x = r / s and t = e / (s h2)
 * (s = RMS of the r crop) to device FP32 [B][D^3] buffers and keeps the
 * target's two norms for pic_cnn_loss. */
int pic_cnn_make_batch(pic_ctx *c, const double *r, const double *a, const double *b, const int *origins_host,
                       int B, int D, float *x, float *t, double h2);
/* Loss of the last batch, mean over crops of E(d)/E(t) + |A_I d|^2/|A_I t|^2
 * with d = y - t: E(d) is the sum of squared differences of d across the
 * grid edges inside the crop's valid interior (cells at least 4 from every
 * face; d^T A d there, the norm CG minimises) and A_I d the 7-point stencil
 * 6 d_i - sum of neighbours on the cells at least 5 from every face (the
 * residual norm). Writes the loss to *loss_host and its gradient with respect
 * to y to gy (device FP32 [B][D^3]). */
int pic_cnn_loss(pic_ctx *c, const float *y, const float *t, int B, int D, float *gy, double *loss_host);

/* ------------------------------------------------------------------------
 * Training of the network behind one call. The paper has no learned part;
 * this follows the learned-preconditioner pattern the library adds to the
 * PCG solve of Sec. 3.2: (residual, error) pairs, random crops, the loss of
 * pic_cnn_loss, Adam, and selection of the kept weights by the flexible-CG
 * iterations of a held-out solve.
 *   PIC_TRAIN_PRECONDITIONER: the pairs come from the library's own FP64
 *     Jacobi-PCG solves of the CIC deposits of `sets` seeded Landau initial
 *     conditions (grid^3 x 8 ppc, seeds seed .. seed + sets - 1): the
 *     converged phi* (tol 1e-12) and the iterates after 1, 2, 4, ..., 128
 *     iterations from zero; scored by PIC_PC_CNN solves.
 *   PIC_TRAIN_SMOOTHER: white-noise errors e (Philox4x32-10 normals, seeds
 *     as above) and r = A e, for the finest-level smoother of the multigrid
 *     V-cycle (PIC_PC_MG_CNN); scored by PIC_PC_MG_CNN solves.
 * Each Adam step draws a set, a snapshot and `batch` crop origins from a
 * Philox4x32-10 stream keyed by `seed` whose counter is the Adam step count,
 * so a training resumed from a weights file (resume = 1, after pic_cnn_load)
 * continues the stream. Without resume the weights start from the Jacobi
 * direction plus seeded noise. With validate_every > 0 the training state is
 * scored every validate_every steps and at the end (flexible CG to rel-res
 * 1e-10 of the CIC deposit of a val_grid^3 x 8 ppc Landau initial condition
 * with seed val_seed), and the best scored state (weights, Adam moments and
 * step count) is the one the context keeps; with 0 the last state is kept.
 * The training runs in contexts of its own on the context's device and
 * stream (the training grid, the validation grid); the context `c` only
 * receives the result, so it may be of any size or a solver-only context.
 * Synchronises. PIC_EINVAL for options out of range (32 <= grid <= 256,
 * grid % 16 == 0, 16 <= crop <= grid, crop % 16 == 0, 1 <= batch, sets <= 64,
 * lr > 0, val_grid % 32 == 0 in [32, 512]); PIC_ESTATE for resume without
 * weights.
 * ------------------------------------------------------------------------ */
enum { PIC_TRAIN_PRECONDITIONER = 0, PIC_TRAIN_SMOOTHER = 1 };
typedef struct {
  int target;          /* PIC_TRAIN_PRECONDITIONER or PIC_TRAIN_SMOOTHER */
  int grid;            /* training grid (64) */
  int sets;            /* training right-hand sides (4) */
  int steps;           /* Adam steps of this call (600) */
  int batch;           /* crops per step (8) */
  int crop;            /* crop edge D (32) */
  double lr;           /* Adam step size (2e-3) */
  uint64_t seed;       /* data, crop-origin and initial-weight seed (11) */
  int validate_every;  /* steps between scorings (100; 0 = keep the last state) */
  int val_grid;        /* validation grid (128) */
  uint64_t val_seed;   /* validation seed (21) */
  int resume;          /* 1 = continue from the context's weights, Adam moments and step */
  int restarts;        /* independent trainings from other initial weights and crop streams
                          (same data), the best validated state kept (1; > 1 needs
                          validate_every > 0 and resume = 0; at most 16) */
} pic_train_opts;
typedef struct {
  int steps;           /* Adam steps taken by this call */
  int adam_steps;      /* Adam step count of the kept state */
  int best_step;       /* step of this call whose state was kept */
  int best_iters;      /* its validation iterations (-1 without validation) */
  int best_restart;    /* the restart it came from */
  double loss_first;   /* mean loss of the first 10 steps */
  double loss_last;    /* mean loss of the last 50 steps */
  double seconds;      /* wall time of the call */
} pic_train_info;
int pic_cnn_train(pic_ctx *c, const pic_train_opts *o, pic_train_info *info);

/* The network's training state in a file: a 32-byte header (magic
 * "PICCNN1\n", format version 1, weight count, Adam step count, FNV-1a
 * 64-bit hash of the payload) and the payload of FP32 master weights, Adam's
 * m and v (PIC_CNN_WEIGHTS floats each, little-endian). pic_cnn_load
 * restores all of it (so training can resume) and rebuilds the inference
 * kernels; PIC_EINVAL for an unreadable, truncated, foreign or corrupted
 * file, PIC_ESTATE from pic_cnn_save without weights. Both synchronise. */
int pic_cnn_save(pic_ctx *c, const char *path);
int pic_cnn_load(pic_ctx *c, const char *path);

/* Arithmetic of the training passes (pic_cnn_forward, pic_cnn_backward):
 * PIC_CNN_TRAIN_BF16 (default) runs the convolutions on the tensor cores
 * with BF16 weights and activations and FP32 accumulation;
 * PIC_CNN_TRAIN_FP32 is a test mode that runs every convolution of both
 * passes on the CUDA cores in FP32 (FP32 activations and data gradients,
 * the FP32 master weights), so that the gradients can be compared with an
 * FP64 reference element by element. A backward pass must follow a forward
 * pass in the same mode (PIC_ESTATE otherwise). PIC_EINVAL for another mode. */
enum { PIC_CNN_TRAIN_BF16 = 0, PIC_CNN_TRAIN_FP32 = 1 };
int pic_cnn_set_train_precision(pic_ctx *c, int mode);

/* One convolution of the packed network without epilogue, for tests: which =
 * 0..3 forward layers 1..4, 4..6 data-gradient convs of layers 4, 3, 2.
 * Input: FP32 [B][D^3] for which 0 and 4, else BF16 [B][D^3][16]; output FP32
 * [B][D^3][16] (accumulator as is). */
int pic_cnn_conv_raw(pic_ctx *c, int which, const void *in, float *out, int B, int D);

/* Profiling (tracing of device time, no effect on results). While enabled,
 * the library records CUDA events on the context stream around every public
 * call (per phase) and around a sample of the solver's kernel launches (the
 * first iteration of every status-check batch), and counts every kernel it
 * launches. Read and optionally reset the totals with pic_profile_read
 * (synchronises the stream). */
enum { PIC_PHASE_DEPOSIT = 0, PIC_PHASE_SOLVE = 1, PIC_PHASE_PUSH = 2, PIC_PHASE_ENERGY = 3, PIC_NPHASE = 4 };
/* Sampled kernels: the CG direction and update kernels, the whole
 * preconditioner application (learned kernel or V-cycle), flexible CG's dot
 * products, and the finest-level kernels of the multigrid V-cycle (two-sweep
 * pre-smoothing, residual, restriction, prolongation + first post-sweep,
 * second post-sweep; with the learned smoother the residual after the
 * prolongation counts as the prolongation slot), the particle kernels and the
 * particle-in-Fourier spreading and interpolation kernels (every launch). */
enum {
  PIC_KER_PAP = 0, PIC_KER_UPDATE = 1, PIC_KER_PRECOND = 2, PIC_KER_DOT = 3,
  PIC_KER_MG_PRE = 4, PIC_KER_MG_RESID = 5, PIC_KER_MG_RESTRICT = 6, PIC_KER_MG_PROLONG_SMOOTH = 7,
  PIC_KER_MG_SMOOTH = 8,
  PIC_KER_SCATTER = 9,  /* the sort's record scatter (every pic_deposit that sorts) */
  PIC_KER_DEPOSIT = 10, /* the two deposit passes (cells, then nodes) */
  PIC_KER_PUSH = 11,    /* the gather + push kernel */
  PIC_KER_PIF_SPREAD = 12, /* particle-in-Fourier: spreading the charges to the oversampled grid */
  PIC_KER_PIF_GATHER = 13, /* particle-in-Fourier: interpolating one field component (3 per field) */
  PIC_NKER = 14
};
typedef struct {
  int64_t launches;           /* kernels launched by the context (counted always) */
  int phase_calls[PIC_NPHASE];
  double phase_ms[PIC_NPHASE];
  int ker_samples[PIC_NKER];  /* sampled launches of each PIC_KER_* kernel */
  double ker_ms[PIC_NKER];    /* their total device time */
  int ker_precision[PIC_NKER]; /* PIC_PREC_* of the sampled launches (last solve) */
} pic_profile_stats;

int pic_profile_enable(pic_ctx *c, int on);
int pic_profile_read(pic_ctx *c, pic_profile_stats *out, int reset);

/* Field energy for callers that cannot allocate device memory (this entry
 * point has no counterpart in the paper). It needs no pic_ctx: the caller
 * passes `phi` (device FP64 [N^3], x fastest, 16-byte aligned), the grid size
 * N (8 <= N <= 1024, N % 8 == 0; larger sizes return PIC_EINVAL) and the
 * wavenumber k (L = 2 pi / k), and receives out_w[d] = h^3 sum_i E_{d,i}^2,
 * d = x, y, z, in `out_w` (device memory, 3 doubles), written asynchronously
 * on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 * It calls no cudaMalloc, cudaFree or other allocating routine. Its reduction
 * scratch is a fixed 48.25 KiB file-scope device array that every GPU loading
 * the library keeps until exit; all calls on a device share it, so calls that
 * overlap on the GPU (different streams) race and must be serialised by the
 * caller. Every call looks up the array's device address in the current
 * device's context (cudaGetSymbolAddress, which allocates nothing); the first
 * call on a device also loads the library's module there, so make it before
 * any stream capture. Returns PIC_OK, PIC_EINVAL or PIC_ECUDA. */
int pic_field_energy_noalloc(const double *phi, int N, double k, double *out_w, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
