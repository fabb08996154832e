/*
 * ibpme.h -- C ABI of the GB300 immersed-boundary PME library.
 *
 * The library evaluates the regularized, spectrally accurate particle-mesh
 * Ewald sums of Krucker-Velasquez, Swan & Sherman, "Immersed boundary method
 * for dynamic simulation of polarizable colloids of arbitrary shape in
 * explicit ion electrolytes" (arXiv:2401.04865), Sec. III.D, and uses them
 * as the matrix-vector product of the induced-charge saddle system of
 * Sec. III.B (Eq. saddle), the bead forces of Sec. III.C (Eq. beadforce)
 * and the Brownian-dynamics step of Sec. V.A.
 *
 * Conventions shared by every entry point:
 *   - Arrays are plain pointers to IEEE double (or int32 where stated),
 *     row-major.  A pointer may address device memory or host memory: the
 *     library asks the CUDA driver which it is and stages host arrays through
 *     its own device buffers (the copies run on the context stream).
 *   - Positions x are [n][3]; they may lie anywhere (they are wrapped into the
 *     periodic box internally).  Charges q are [nrhs][n].
 *   - Potentials are psi_alpha - psi_0(x_alpha) (Eq. pot_charge), fields are
 *     E = -grad psi, in units where the fluid permittivity is eps_f.
 *   - Bodies are contiguous ranges of beads given by CSR offsets (Appendix,
 *     summation tensor Sigma); an ion is a body of one bead (Sec. III.B).
 *   - Ownership: the caller owns every array; the library never keeps a
 *     pointer after a call returns.  The context owns its device scratch.
 *   - Streams: all work is enqueued on the context stream.  Entry points that
 *     return results in host memory, and induced_charge_solve (which needs its
 *     convergence flag), synchronize that stream before they return.
 *   - Errors: every entry point returns an ibpme_status and never throws;
 *     ibpme_last_error() gives a message for the calling thread.  After an
 *     error the outputs are unspecified.
 *   - All beads share one radius a (Sec. III.A).
 *   - Environment switches (read when the data they govern are built; for
 *     diagnostics and tests, results agree to rounding either way):
 *     IBPME_NO_GRAPHS (no captured iteration graphs), IBPME_NO_TILES (no
 *     shared-memory tiles in spreading and gathering), IBPME_NO_COMPACT (every
 *     intra-body pair in the real-space table), IBPME_VERBOSE (solver log).
 */
#ifndef IBPME_H
#define IBPME_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibpme_ctx ibpme_ctx;

#define IBPME_MAX_RADIUS_CLASSES 4

typedef enum {
    IBPME_OK = 0,
    IBPME_ERR_ARG = 1,            /* invalid argument (sizes, box, mesh < P, r_cut >= L/2, ...) */
    IBPME_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    IBPME_ERR_CUFFT = 3,          /* a cuFFT call failed */
    IBPME_ERR_OOM = 4,            /* device allocation failed */
    IBPME_ERR_NOT_CONVERGED = 5,  /* the Krylov solve hit max_iter; outputs hold the last iterate */
    IBPME_ERR_UNEQUAL_RADII = 6,  /* the call does not take beads of unequal radii (radius classes):
                                     the batched solve and the learned warm start */
    IBPME_ERR_TIMEOUT = 7,        /* a bounded device wait ran out: the tensor cores of the
                                     learned guess, or the tensor (TMA) copies of a tiled mesh
                                     gather (reported after the gather's stream synchronised:
                                     by that call, or by the context's next call) */
    IBPME_ERR_NONFINITE = 8       /* NaN/Inf in an input or in the iteration */
} ibpme_status;

enum { IBPME_FP64 = 0,            /* every step in FP64 */
       IBPME_MIXED = 1 };         /* FP32 mesh (spread, FFT, scale, gather), FP64 near field and
                                     Krylov; inside a solve the corrections come from an inner
                                     operator whose near field is FP32 too, refined against the
                                     FP64 operator.  At rtol >= 1e-7 the first residual of a
                                     nonzero guess takes the FP32 mesh; every residual that
                                     decides convergence takes the FP64 operator */

/* Parameters of the spectral Ewald split (Sec. III.D).  A zero in a field
 * marked "auto" asks pme_setup to derive it with the rules of Sec. III.D.2:
 *   k_c = pi (N_g - 1) / L          (from N_g = 1 + L k_c / pi, smallest axis)
 *   xi  = k_c / (2 sqrt(ln(1/tol))) (wave-space bound e^{-k_c^2/4xi^2} = tol)
 *   r_cut = sqrt(ln(1/tol)) / xi + 2a (real-space bound, Eq. realspaceerror)
 *   P   = ceil(2 ln(1/tol) / pi)    (contraction bound e^{-pi P/2} <= tol, Eq. contractionerror)
 *   eta = h^2 xi^2 P / pi           (h = largest L_d / N_d)
 * If mesh is {0,0,0}, xi must be given and N_g = 1 + L k_c/pi with
 * k_c = 2 xi sqrt(ln(1/tol)), rounded up to a size with prime factors 2, 3, 5, 7. */
typedef struct {
    double box[3];        /* periodic box side lengths L_x, L_y, L_z (> 0) */
    int mesh[3];          /* grid points per axis N_x, N_y, N_z (>= P), or 0 = auto */
    double xi;            /* Ewald splitting parameter, 0 = auto */
    double eta;           /* spectral-Ewald Gaussian split, 0 = auto */
    double r_cut;         /* real-space cutoff, 0 = auto; must be < L/2 */
    int P;                /* stencil points per axis (<= 32), 0 = auto */
    double tol;           /* accuracy target of the automatic rules (e.g. 1e-6); 0 -> 1e-6 */
    double bead_radius;   /* a, shared by all beads (> 0); ignored with radius classes, where
                             ibpme_get_params reports the largest class radius */
    double eps_f;         /* fluid permittivity (> 0); eps_f = 1/(4 pi l_B) with kT = 1 */
    int precision;        /* IBPME_FP64 or IBPME_MIXED */
    int max_rhs;          /* largest nrhs a call will pass (1..8); 0 -> 3 */
    int n_radius_classes; /* 0 or 1: every bead has bead_radius; 2..IBPME_MAX_RADIUS_CLASSES:
                             beads of unequal radii, bead b of radius class_radius[cls[b]]
                             with cls bound by ibpme_set_radius_classes */
    double class_radius[IBPME_MAX_RADIUS_CLASSES];   /* radii of the classes (> 0) */
} ibpme_params;

/* Create a context: resolves the automatic parameters, allocates the meshes
 * (FP64, plus FP32 in mixed precision), builds cuFFT plans and the k-space
 * Green's-function table of Sec. III.D.2 (Eq. after H_hat).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  On error *ctx is NULL. */
ibpme_status pme_setup(ibpme_ctx** ctx, const ibpme_params* params, void* cuda_stream);

/* Free the context and all its device memory.  NULL is accepted. */
ibpme_status pme_destroy(ibpme_ctx* ctx);

/* Change the stream on which later calls enqueue their work. */
ibpme_status ibpme_set_stream(ibpme_ctx* ctx, void* cuda_stream);

/* Copy the resolved parameters (all "auto" fields filled in) to *out. */
ibpme_status ibpme_get_params(const ibpme_ctx* ctx, ibpme_params* out);

/* Beads of unequal radii (the paper fixes one radius, Sec. III.A; this is its
 * direct extension).  A bead of radius a carries its charge on a shell whose
 * transform is j0(ka), so beads alpha and beta interact through
 *     M_hat(k) = j0(k a_alpha) j0(k a_beta) / (eps k^2)
 * in place of j0^2(ka)/(eps k^2) of Eq. M00_Fourier.  The library spreads each
 * class into its own mesh channel, combines the transformed channels with
 * j0(k a_c) j0(k a_d), gathers each bead from its own class's channel, and gives
 * every pair within r_cut its two-radius real-space kernel (the average of
 * erfc(xi s)/(4 pi eps s) over both shells), every bead its own class's self term;
 * the auto r_cut uses the largest class radius; the body-block preconditioner
 * and the hard-sphere forces of ibpme_bd_advance (contact at a_alpha + a_beta)
 * take the bead radii too.
 *   n    number of beads of the calls that follow (>= 0); 0 unbinds
 *   cls  host array [n] of class indices in 0 .. n_radius_classes - 1, copied
 * A context created with n_radius_classes >= 2 needs a binding for the bead
 * count of every call (IBPME_ERR_ARG otherwise); positions may change between
 * calls, classes stay with the bead index.  induced_charge_solve_batch and
 * the learned guesses return IBPME_ERR_UNEQUAL_RADII on such a context.
 * IBPME_ERR_ARG if the context has no radius classes or an index is out of range. */
ibpme_status ibpme_set_radius_classes(ibpme_ctx* ctx, int n, const int* cls);

/* Hydrodynamic mobility with the Rotne-Prager-Yamakawa tensor: the interactions the
 * paper neglects and names as the way to add them (Sec. V.A, Eq. velocity):
 *     U_alpha = sum_beta M^H_alpha_beta . F_beta,
 * M^H the RPY tensor of beads of radius bead_radius in a fluid of viscosity mu, i.e.
 * the Oseen tensor averaged over both beads' surfaces, M_hat(k) = j0^2(ka)(I - k_hat
 * k_hat)/(mu k^2), summed over the periodic images with the k = 0 mode left out.
 * Computed with the context's spectral-Ewald split (xi, mesh, P, r_cut) under
 * Hasimoto's weight (1 + k^2/(4 xi^2)) e^{-k^2/(4 xi^2)}: the three force components
 * spread, transformed, projected and gathered like three right-hand sides, the real
 * space from a table of the two radial functions of M_RPY minus the wave kernel.
 * The mesh runs in the context's precision (FP32 in IBPME_MIXED), the real space in FP64.
 *   n    number of beads (>= 0)
 *   x    [n][3] positions; F [n][3] forces; U [n][3] velocities (output, overwritten)
 *   mu   viscosity (> 0)
 * Pointers may be host or device memory (host outputs are written when the call
 * returns).  IBPME_ERR_ARG for a NULL pointer with n > 0 or mu <= 0;
 * IBPME_ERR_UNEQUAL_RADII on a context with radius classes. */
ibpme_status ibpme_rpy_mobility(ibpme_ctx* ctx, int n, const double* x, const double* F, double mu, double* U);

/* Message of the last error raised on the calling thread ("" if none). */
const char* ibpme_last_error(void);

/* Spreading, Sec. III.D.2 Eq. H_hat and step 2 of Sec. III.D.3:
 *   H(x_g) = (2 xi^2/(pi eta))^{3/2} sum_beta q_beta exp(-2 xi^2 |x_g - x_beta|^2 / eta)
 * on the grid nodes x_g = (i h_x, j h_y, k h_z), each bead restricted to the
 * P closest nodes per axis (first node floor(x/h - P/2) + 1, periodic).
 *   n      number of beads (>= 0)
 *   x      [n][3] positions; q [nrhs][n] charges; 1 <= nrhs <= max_rhs
 *   grid_out  NULL, or [nrhs][N_z][N_y][N_x] of the context precision's
 *          real type (double for IBPME_FP64, float for IBPME_MIXED), x fastest.
 * The grid stays in the context for inspection; it is overwritten by the next call. */
ibpme_status pme_spread(ibpme_ctx* ctx, int n, const double* x, const double* q, int nrhs, void* grid_out);

/* One PME evaluation, Sec. III.D.3 steps 1-6: psi = M q for every bead
 * (real-space sum with the cell list + self term + spread, FFT, Green's-function
 * scaling, inverse FFT, trapezoid-rule gather), optionally the field.
 *   psi  [nrhs][n] (required), E [nrhs][n][3] or NULL.
 * The near field is computed in FP64; the mesh in the context precision. */
ibpme_status pme_field(ibpme_ctx* ctx, int n, const double* x, const double* q, int nrhs,
                       double* psi, double* E);

/* Bodies for the saddle system (Sec. III.B, Appendix). */
typedef struct {
    int n_bodies;              /* N_b >= 1 */
    const int* body_offsets;   /* [N_b + 1] int32 CSR offsets into the beads, offsets[0] = 0,
                                  offsets[N_b] = n, every body non-empty */
    const double* X;           /* [N_b][3] body reference points (centre of mass, Sec. III.B) */
    const double* Q;           /* [N_b] net body charges (Eq. Q_tot) */
} ibpme_bodies;

/* Initial guesses.  LEARNED: the learned warm start g (below).  LEARNED_STEP, for a
 * sequence of calls on the same bodies (a trajectory): q_out holds on input the
 * converged charges of the previous call and the guess is q + g(now) - g(previous),
 * the learned change added to them, with g(previous) the learned guess that call
 * left in the context; a call without one (the first, or after the body structure,
 * bead count or field count changed) starts from g(now).  Both keep g(now) for the
 * next call. */
enum { IBPME_GUESS_ZERO = 0, IBPME_GUESS_USER = 1, IBPME_GUESS_LEARNED = 2, IBPME_GUESS_LEARNED_STEP = 3 };

typedef struct {
    double rtol;        /* target relative residual of Eq. saddle, ||b - A u|| / ||b||; 0 -> 1e-6 */
    int restart;        /* GMRES restart length m (1..128); 0 -> 50 */
    int max_iter;       /* cap on Krylov iterations (all restarts, all refinement steps); 0 -> 3000 */
    int guess;          /* IBPME_GUESS_*; USER reads q_out as the initial charges.  The initial
                           body potentials are always the least-squares fit to the initial
                           charges (mean over each body of (M q)_j - r_j.E0) */
    const void* mlp;    /* trained ibpme_mlp (IBPME_GUESS_LEARNED[_STEP]), else NULL */
    int precision;      /* -1 = context precision, else IBPME_FP64 / IBPME_MIXED (mixed needs a
                           mixed context) */
    int precond;        /* IBPME_PRECOND_BODY (0, the default) or IBPME_PRECOND_NONE */
} ibpme_solve_opts;

/* Right preconditioner of the Krylov iteration (not in the paper; the converged
 * solution and its FP64 residual test are the same either way).  BODY applies,
 * for every multi-bead body, the exact inverse of the body's own saddle block with
 * the free-space kernel of Sec. II, [-M_b e; e^T 0]^{-1}, and the identity to the
 * rest; a configuration with a body of more than 1,024 beads is left
 * unpreconditioned.  M_b depends only on
 * the distances between a rigid body's beads, so the inverses are computed once
 * per body shape (FP64 Gauss-Jordan on the device, kept in FP32) and cached in
 * the context; identical bodies share one. */
enum { IBPME_PRECOND_BODY = 0, IBPME_PRECOND_NONE = 1 };

typedef struct {
    int iters;              /* Krylov iterations (operator applications inside GMRES) */
    int outer;              /* refinement steps (mixed precision), 1 for FP64 */
    int matvecs_fp64;       /* FP64 operator applications (true residuals, RHS) */
    double rel_residual;    /* final ||b - A u||_2 / ||b||_2 with the FP64 operator, worst RHS */
    double time_ms;         /* host wall time of the call (device outputs complete in stream order) */
    int fell_back;          /* 1 if the learned guess was rejected for the zero guess */
    double init_rel_residual;   /* ||b - A u0|| / ||b|| of the initial guess actually used (FP64
                                   operator; FP32 mesh where the first residual takes it) */
} ibpme_solve_stats;

/* Induced-charge solve, Sec. III.B Eq. saddle:
 *   [-M  Sigma^T] [q          ]   [-r . E0]
 *   [Sigma    0 ] [Psi - Psi_0] = [   Q   ],   r_ij = x_ij - X_i (minimum image)
 * by restarted GMRES with every vector and scalar on the device.  Single-bead
 * bodies (ions) have q = Q fixed; they are eliminated exactly and their
 * Psi - Psi_0 is recovered with one FP64 evaluation.  Convergence is decided
 * on the full system with the FP64 operator.
 *   E0       [nrhs][3] external field per right-hand side
 *   q_out    [nrhs][n] bead charges (initial guess on input when guess = USER)
 *   psi_out  [nrhs][N_b] Psi - Psi_0 per body, or NULL
 *   S_out    [nrhs][N_b][3] body dipoles S_i = sum_j r_ij q_ij (Eq. rigid_dipole), or NULL
 *   stats    or NULL
 * Returns IBPME_ERR_NOT_CONVERGED (with the last iterate written) if max_iter is hit. */
ibpme_status induced_charge_solve(ibpme_ctx* ctx, int n, const double* x, const ibpme_bodies* bodies,
                                  const double* E0, int nrhs, const ibpme_solve_opts* opts,
                                  double* q_out, double* psi_out, double* S_out,
                                  ibpme_solve_stats* stats);

/* Batched configurations: n_configs independent systems of Eq. saddle solved in
 * one call (not in the paper, which solves one system at a time; its
 * polarizability tensors of Sec. IV need three field directions per shape).
 * Configuration k owns the bodies cfg_bodies[k] .. cfg_bodies[k+1]-1 and hence a
 * contiguous range of beads; each lives in its own periodic copy of the context's
 * box with the context's bead radius and permittivity.  Beads of different
 * configurations never interact: no real-space pairs, separate mesh channels,
 * separate k = 0 sums.  Every PME evaluation serves all configurations and all
 * right-hand sides at once (nrhs * n_configs mesh channels, one batched FFT),
 * and each (configuration, right-hand side) pair is its own GMRES system with
 * its own Hessenberg matrix and convergence test.
 *   cfg_bodies  HOST int32 [n_configs + 1], cfg_bodies[0] = 0, cfg_bodies[n_configs]
 *               = bodies->n_bodies, strictly increasing (no empty configuration)
 *   E0          [nrhs][3], the same fields for every configuration
 *   q_out, psi_out, S_out  as for induced_charge_solve over all n beads / N_b bodies
 *   stats       [n_configs] or NULL: per configuration, the worst right-hand side;
 *               iteration counts are those of the common loop
 * guess = IBPME_GUESS_LEARNED or IBPME_GUESS_LEARNED_STEP is not accepted here (IBPME_ERR_ARG).
 * Returns IBPME_ERR_NOT_CONVERGED if any configuration misses rtol. */
ibpme_status induced_charge_solve_batch(ibpme_ctx* ctx, int n, const double* x, const ibpme_bodies* bodies,
                                        int n_configs, const int* cfg_bodies, const double* E0, int nrhs,
                                        const ibpme_solve_opts* opts, double* q_out, double* psi_out,
                                        double* S_out, ibpme_solve_stats* stats);

/* Forces and torques, Sec. III.C:
 *   f_alpha = q_alpha E0 - 1/2 (grad_alpha M) : q q = q_alpha (E0 + E_alpha)   (Eq. beadforce)
 *   F_i = sum_j f_ij,  L_i = sum_j r_ij x f_ij
 *   U = 1/2 sum_i (Q_i Psi_i - S_i . E0), Psi_i = (Psi - Psi_0)_i - X_i . E0   (Eq. pot_syst)
 * where E_alpha is the PME field of all charges at bead alpha (one spread, one
 * FFT pair, a gradient gather and the real-space gradient), q a converged
 * solution and E0 one field [3].  Q is taken from bodies->Q.
 *   f_bead [n][3] or NULL; F, L [N_b][3] required; U [1] or NULL. */
ibpme_status body_force_torque(ibpme_ctx* ctx, int n, const double* x, const double* q,
                               const ibpme_bodies* bodies, const double* E0,
                               double* f_bead, double* F, double* L, double* U);

/* Brownian dynamics, Sec. V.A. */
typedef struct {
    double dt;                    /* time step (> 0) */
    double gamma;                 /* drag coefficient of one bead (> 0) */
    double kT;                    /* thermal energy (>= 0; 0 = deterministic) */
    unsigned long long seed;      /* Philox4x32-10 key */
    long long step;               /* step counter (part of the Philox counter) */
} ibpme_bd_params;

/* Grand capacitance tensor of Sec. III.B, Eq. QS_capacitance:
 *     [Q; S] = C [Psi - Psi_0; E0],   C = Sigma' M^{-1} Sigma'^T,
 * for the bodies at x, with E0 the field of each body's own bead rows.  C is
 * 4 N_b x 4 N_b, rows and columns ordered [Q_1 .. Q_Nb, S_1x, S_1y, S_1z, S_2x, ...]
 * (body-major dipole rows).  Column k holds the body charges and dipoles of the
 * charges q = M^{-1} psi_k, where psi_k (column k of Sigma'^T) is 1 on the beads of
 * body k (k < N_b) or r_ij,d on the beads of body i (k = N_b + 3 i + d) and 0
 * elsewhere; the 4 N_b systems M q = psi_k are solved by the Krylov solver of
 * induced_charge_solve (options as there: rtol on ||psi_k - M q|| / ||psi_k||,
 * precision, body-block preconditioner) in groups of at most max_rhs right-hand
 * sides, from the zero guess.  C is symmetric positive definite up to the
 * tolerance.  With one sphere per periodic cell, C_SE / (eps_f V) gives the
 * lattice's effective permittivity eps_eff / eps_f - 1 (Sec. IV.C).
 *   bodies   every body needs two beads or more (IBPME_ERR_ARG otherwise: single
 *            beads are not conductors here); bodies->Q is not used and may be NULL
 *   opts     NULL = defaults; guess must be IBPME_GUESS_ZERO
 *   C_out    [4 N_b][4 N_b] row-major, device or host
 *   stats    the worst residual and most iterations over the groups, or NULL
 * Returns IBPME_ERR_NOT_CONVERGED (C written) if a group misses rtol. */
ibpme_status ibpme_capacitance(ibpme_ctx* ctx, int n, const double* x, const ibpme_bodies* bodies,
                               const ibpme_solve_opts* opts, double* C_out, ibpme_solve_stats* stats);

/* One Euler-Maruyama step (Eq. forward) with free-draining mobility M^H = I/gamma.
 * The bead forces f_bead [n][3] are augmented by the Heyes-Melrose hard-sphere
 * pair forces of Eq. hardsphereFD (beads of different bodies closer than 2a).
 * Ions: dx = F dt/gamma + sqrt(2 kT dt/gamma) n.  Rigid bodies: U = F_i/(N_i gamma),
 * Omega = (gamma J_i)^{-1} L_i, J_i = sum_j (|r_ij|^2 I - r_ij r_ij^T), Brownian
 * displacements with covariance 2 kT dt times the same mobilities; beads move
 * rigidly with the body.  Normals: Philox4x32-10 on counter
 * (body, step, t, 0x1B5EED), key (seed lo, seed hi), Box-Muller on the first two words.
 *   x_out [n][3] new positions, X_out [N_b][3] new reference points (may alias x / bodies->X
 *   only if they are device pointers). */
ibpme_status ibpme_bd_step(ibpme_ctx* ctx, int n, const double* x, const ibpme_bodies* bodies,
                           const double* f_bead, const ibpme_bd_params* bd,
                           double* x_out, double* X_out);

/* One step of the Brownian dynamics of Sec. V.A in one call: the induced-charge
 * solve of Eq. saddle at the positions x for one field E0 [3] (options as
 * induced_charge_solve), the bead forces of Eq. beadforce with the body forces,
 * torques and energy of body_force_torque, and the Euler-Maruyama step of
 * ibpme_bd_step with those bead forces.  The positions are checked, the bodies
 * uploaded and the real-space pair table built once for the three parts.  The
 * field of the forces is the gradient gathered from the FP64 mesh of the solve's
 * final FP64 residual (which already holds the transformed potential of the final
 * charges) plus the FP64 near field, and the energy takes that residual's FP64
 * potentials: in an FP64 context the results equal the three separate calls up to
 * rounding; in a mixed context the forces carry the FP64 mesh where
 * body_force_torque takes the FP32 mesh.
 *   q_io     [n] bead charges: the initial guess on input when opts->guess = USER,
 *            the solution on output
 *   psi_out  [N_b] Psi - Psi_0 per body, or NULL
 *   f_bead   [n][3] bead forces without the hard-sphere part, or NULL
 *   F, L     [N_b][3] body forces and torques;  U [1] energy, or NULL
 *   x_out, X_out, bd  as ibpme_bd_step
 *   stats    the solve's statistics, or NULL
 * Returns IBPME_ERR_NOT_CONVERGED (charges and psi written, forces and positions
 * not) if the solve hits max_iter. */
ibpme_status ibpme_bd_advance(ibpme_ctx* ctx, int n, const double* x, const ibpme_bodies* bodies,
                              const double* E0, const ibpme_solve_opts* opts, const ibpme_bd_params* bd,
                              double* q_io, double* psi_out, double* f_bead, double* F, double* L, double* U,
                              double* x_out, double* X_out, ibpme_solve_stats* stats);

/* ---- Learned warm start (not in the paper) ----
 *
 * A small network (IBPME_MLP_IN features -> 64 -> 64 -> 1, tanh, FP32) maps
 * per-bead features to a first guess of the induced charge of beads on
 * multi-bead bodies.  The features need no mesh evaluation: they come from the
 * bodies' geometry, the field E0, the net charges and the free-space potential
 * and field of the other bodies' fixed charges near the body, so the solve's
 * first residual is the one evaluation a zero guess makes.
 * For bead j of body b with N >= 2 beads, relative positions r from the body's
 * reference point, R = mean |r| over the body, R_max = max |r|, A = 4 pi R^2 / N,
 * h = sqrt(A):
 *   d1, d6   distances from x_j to the nearest and the k-th nearest other bead of
 *            the body, k = min(6, N - 1);
 *   w_k      = exp(-|x_k - x_j|^2 / h^2) over the body's other beads,
 *            m = sum w (x_k - x_j) / sum w, s2 = sum w |x_k - x_j|^2 / sum w,
 *            C = sum w (x_k - x_j)(x_k - x_j)^T / sum w;
 *   n        = the unit eigenvector of the smallest eigenvalue of C (the normal of
 *            the plane that fits the neighbourhood best), signed so that n . r >= 0;
 *            kappa = -2 (m . n) / s2 (1/R on a sphere, 1/(2 rho) on a cylinder);
 *   phi, Es  potential and field at x_j of the fixed charges q_beta (an ion's own
 *            charge, Q/N on a bead of another multi-bead body) of every bead beta
 *            of another body within R_max + 6R of the body's reference point
 *            (minimum image), with the regularised free-space kernel of Sec. II
 *            (1/(4 pi eps r) for r >= 2a, (4a - r)/(16 pi eps a^2) below);
 *   <.>      body means; S = eps A (|E0| + rms |Es|).
 *   f0 = eps A (E0 . n) / S          f1 = eps A |E0 - (E0 . n) n| / S
 *   f2 = eps A (r . E0 - <r . E0>) / (R S)
 *   f3 = eps A (phi - <phi>) / (R S)  f4 = eps A (Es . n) / S
 *   f5 = eps A |Es - (Es . n) n| / S  f6 = kappa R      f7 = |r| / R - 1
 *   f8 = Q / (N S) clipped to +-10   f9 = 10 a / R      f10 = d1 / h
 *   f11 = (d6 - d1) / h.
 * Geometry is taken in FP32; body sums and scales in FP64.  The guess is
 * q = Q/N + S y, then shifted body by body so that sum q = Q exactly (a body with
 * S = 0 gets Q/N).  The network is trained on converged solves (ibpme_mlp_train);
 * the solve uses it with IBPME_GUESS_LEARNED and falls back to the zero guess
 * (stats.fell_back = 1) if its residual is not smaller than |b|.
 * Parameter layout (floats): W1[64][IN], b1[64], W2[64][64], b2[64], W3[64], b3. */
#define IBPME_MLP_IN 12
#define IBPME_MLP_HIDDEN 64
#define IBPME_MLP_NPARAM (IBPME_MLP_HIDDEN * IBPME_MLP_IN + IBPME_MLP_HIDDEN + IBPME_MLP_HIDDEN * IBPME_MLP_HIDDEN + \
                          IBPME_MLP_HIDDEN + IBPME_MLP_HIDDEN + 1)
typedef struct ibpme_mlp ibpme_mlp;

/* New network on the current device, weights N(0, 1/fan_in) from seed, biases 0. */
ibpme_status ibpme_mlp_create(ibpme_mlp** mlp, unsigned long long seed);
ibpme_status ibpme_mlp_destroy(ibpme_mlp* mlp);
/* Copy the IBPME_MLP_NPARAM parameters out / in (host or device pointer); set resets Adam. */
ibpme_status ibpme_mlp_get(const ibpme_mlp* mlp, float* params);
ibpme_status ibpme_mlp_set(ibpme_mlp* mlp, const float* params);
/* y[i] = net(feat[i]) for n samples; feat [n][IBPME_MLP_IN], y [n], device pointers.
 * FP32 throughout on the CUDA cores (the reference of the training kernels). */
ibpme_status ibpme_mlp_forward(ibpme_mlp* mlp, int n, const float* feat, float* y, void* cuda_stream);
/* The same network with the hidden 64 x 64 layer on the tensor cores (tcgen05.mma,
 * BF16 activations and weights, FP32 accumulation in tensor memory); the input and
 * output layers stay FP32.  This is the path of IBPME_GUESS_LEARNED.  Synchronizes
 * the stream; IBPME_ERR_TIMEOUT if a bounded wait for the tensor cores ran out. */
ibpme_status ibpme_mlp_forward_tc(ibpme_mlp* mlp, int n, const float* feat, float* y, void* cuda_stream);
/* Gradient of the mean squared error L = (1/n) sum (net(feat_i) - target_i)^2 with
 * respect to the parameters (grad [IBPME_MLP_NPARAM], host or device) and L. */
ibpme_status ibpme_mlp_gradient(ibpme_mlp* mlp, int n, const float* feat, const float* target, float* grad,
                                float* loss, void* cuda_stream);
/* Adam (lr, beta1 0.9, beta2 0.999) on the mean squared error over shuffled
 * mini-batches of `batch` samples for `epochs` passes; loss_out gets the last
 * epoch's mean batch loss.  feat, target: device arrays. */
ibpme_status ibpme_mlp_train(ibpme_mlp* mlp, int n, const float* feat, const float* target, int batch, int epochs,
                             float lr, unsigned long long seed, float* loss_out, void* cuda_stream);
/* The features above for every bead and field: feat [nrhs][n][IBPME_MLP_IN]
 * (zeros for single-bead bodies).  If q [nrhs][n] (converged charges) and target
 * [nrhs][n] are given, also the training targets y = (q - Q/N) / S (0 on
 * single-bead bodies).  Device pointers only. */
ibpme_status ibpme_features(ibpme_ctx* ctx, int n, const double* x, const ibpme_bodies* bodies, const double* E0,
                            int nrhs, float* feat, const double* q, float* target);

/* ---- Spreading without device allocation (no counterpart in the paper) ----
 *
 * For callers that cannot allocate device memory: code running while a stream
 * is captured into a CUDA graph (where cudaMalloc is not allowed), engines whose
 * device memory belongs to a pool or a framework, and loops that must never reach
 * the allocator.  pme_spread needs a context, which allocates; this variant does
 * the same spreading as pme_spread (same stencil and normalisation) with no context
 * and no allocation of any kind: its only scratch, the positions wrapped into the
 * box, lives in a fixed array inside the library (IBPME_NOALLOC_MAX_BEADS x 3
 * doubles = 6 MiB), which every GPU that loads the library keeps until the
 * process exits.
 *   params   parameters as for pme_setup (resolved on the host, same rules);
 *            params->precision picks the grid type (double or float)
 *   n        0 .. IBPME_NOALLOC_MAX_BEADS beads (larger n: IBPME_ERR_ARG)
 *   x, q     device arrays [n][3], [nrhs][n]; 1 <= nrhs <= 8
 *   grid_out device array [nrhs][N_z][N_y][N_x]; the call clears it, then spreads
 *   cuda_stream  stream for the work (NULL = legacy default stream)
 * Host pointers are rejected (IBPME_ERR_ARG): staging them would allocate.
 * The first call on a device looks up the scratch array's device address for
 * that device; make that first call before any stream capture.  All calls share
 * the one scratch array and it keeps the last call's contents, so calls that
 * can overlap on the GPU (different streams, or different host threads) race:
 * serialise them. */
#define IBPME_NOALLOC_MAX_BEADS 262144
ibpme_status pme_spread_noalloc(const ibpme_params* params, int n, const double* x, const double* q, int nrhs,
                                void* grid_out, void* cuda_stream);

/* Rigid-body mobility problem of the paper's last equation (the hydrodynamic
 * integrator it hands the body forces and torques to, here with the periodic RPY
 * mobility of ibpme_rpy_mobility): bead constraint forces f and body motions
 * W = (U, Omega) with
 *     M^H f = U_b + Omega_b x r_j   for every bead j of body b (rigid motion),
 *     sum_j f_j = F_b,  sum_j r_j x f_j = L_b,
 * r_j the minimum-image position of bead j relative to X_b.  (The paper writes the
 * system with +Sigma'''^T; its (U, Omega) is minus the motion here.)  A single-bead
 * body moves by U alone: its Omega is returned as 0 and its torque ignored.  Bodies
 * of two or more beads must not be collinear (a rod of beads has no resistance to
 * spinning about its axis, and the system is then singular).  Solved by restarted
 * GMRES (classical Gram-Schmidt twice per step) on the unknowns (f, W), each
 * iteration one RPY mobility product in the context's precision, right-
 * preconditioned by default (opts->precond = IBPME_PRECOND_BODY) with the exact
 * inverse of every multi-bead body's own block under the free-space RPY tensor
 * (an FP32 inverse of its 3 n_b x 3 n_b mobility, built at every call, bodies of
 * up to 2,730 beads; larger ones leave the solve unpreconditioned) and of every
 * single bead's; IBPME_PRECOND_NONE iterates on the bare system.
 *   n, x     beads [n][3]; bodies: n_bodies, body_offsets, X (Q must point to n_bodies
 *            doubles, as for the other calls, but its values are not used)
 *   FL       [n_bodies][6] forces and torques (F, L) per body
 *   mu       viscosity (> 0)
 *   opts     rtol (0 -> 1e-6) on ||b - A z|| / ||b||, restart (0 -> 50, <= 200),
 *            max_iter (0 -> 3000), precond; the other fields are ignored; NULL = defaults
 *   W        [n_bodies][6] output (U, Omega); f_out [n][3] constraint forces or NULL
 *   stats    iters, outer, rel_residual, time_ms (or NULL)
 * In an IBPME_MIXED context the product runs its mesh and real space in FP32 and
 * is exact to about 1e-7, so rtol much below 1e-6 is not reached there.
 * Pointers may be host or device memory.  IBPME_ERR_NOT_CONVERGED when max_iter
 * iterations do not reach rtol (the outputs hold the last iterate);
 * IBPME_ERR_UNEQUAL_RADII on a context with radius classes. */
ibpme_status ibpme_rigid_mobility(ibpme_ctx* ctx, int n, const double* x, const ibpme_bodies* bodies,
                                  const double* FL, double mu, const ibpme_solve_opts* opts, double* W,
                                  double* f_out, ibpme_solve_stats* stats);

/* ---- Instrumentation (no counterpart in the paper) ---- */

/* Number of kernel launches the library has issued in this process (its own
 * kernels, including those replayed from its captured CUDA graphs; cuFFT's
 * launches are not counted). */
long long ibpme_kernel_launches(void);

/* Stages that can be timed: 0 near_build (cell list + pair table), 1 near_apply
 * (real-space SpMV/field), 2 spread, 3 fft_forward, 4 scale, 5 fft_inverse,
 * 6 gather (2-6: FP32 mesh), 7 krylov (Arnoldi/Givens kernels of one iteration),
 * 8 bodies, 9-13 the FP64 mesh (spread64, fft_forward64, scale64, fft_inverse64,
 * gather64), 14 near_apply32 (the FP32 real-space pass of a mixed solve's inner
 * operator), 15 near_field (real-space field of the force pass), 16 rpy_near (the
 * real-space share of ibpme_rpy_mobility).
 * ibpme_profile(mask) enables CUDA-event timing of the stages in the bit mask
 * (0 disables) and resets the totals; each enabled stage then records an event
 * pair on the stream it runs on. */
ibpme_status ibpme_profile(unsigned stage_mask);

/* Synchronizes the device, then writes the accumulated milliseconds and the
 * number of timed launches of the first max_stages stages (either array may be NULL). */
ibpme_status ibpme_profile_read(int max_stages, double* total_ms, long long* launches);

/* Name of a stage ("" if out of range). */
const char* ibpme_stage_name(int stage);

#ifdef __cplusplus
}
#endif

#endif /* IBPME_H */
