/*
 * gpw.h — C ABI of libgpw: multigrid Gaussian-plane-wave (FFTDF) collocation,
 * integration and nuclear-gradient contraction on one GB300 (sm_103a), FP64.
 *
 * The operations follow arXiv 2603.24881 ("Implementation of the multigrid
 * Gaussian-Plane-Wave algorithm with GPU acceleration in PySCF"):
 *   - eval_rho:     density of Eq. (rho), evaluated as Eq. (rho_wrap) (one orbital
 *                   in the home cell, the other over lattice images, folded back),
 *                   pair by pair on the coarsest multigrid level that resolves the
 *                   pair exponent (Sec. II, multigrid), then combined on the finest
 *                   grid by Fourier interpolation;
 *   - eval_mat:     the two-electron Fock matrix of Eq. (J) / (J_wrap) for a given
 *                   real-space potential, integrated on the same levels;
 *   - eval_mat_ip1: the Hxc part of the nuclear gradient (Algorithm 3);
 *   - fock:         rho -> Poisson (Eqs. vH, vHG) + LDA or PBE exchange -> V;
 *   - the kinetic-energy density of meta-GGA functionals, its Fock term and gradient.
 *
 * Conventions
 *   Units: Bohr and Hartree.  Any lattice (rows a1, a2, a3).  Non-orthogonal cells
 *   (App., non-orthogonal lattices) use 4x8x16 sub-boxes for both grid passes.
 *   Shells are Cartesian with angular momentum 0..3; within a shell the AO order is
 *   lexicographic with x^l first (d: xx, xy, xz, yy, yz, zz).  AOs follow the shell
 *   order of the descriptor.
 *   Grids are C order [N0][N1][N2] along a1, a2, a3; point (i0,i1,i2) sits at
 *   (i0/N0) a1 + (i1/N1) a2 + (i2/N2) a3.  Level 0 is the finest grid.
 *   Matrices are row-major nao x nao doubles.
 *
 * Ownership and memory
 *   The caller owns every D, rho, v, V and gradient buffer: device memory, FP64,
 *   contiguous, unless a parameter says "host".  The plan owns its pair tables,
 *   level grids, spectra, cuFFT plans and scratch, all allocated by gpw_plan; the
 *   evaluation calls allocate nothing (gpw_fock_grad_host makes the plan's device
 *   copies of its host buffers on its first call).
 *
 * Streams
 *   Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy default)
 *   except where noted.  One plan may be used by one stream at a time; different
 *   plans are independent.
 *
 * Errors
 *   Every int-returning call returns GPW_OK (0) or a negative GPW_E* code and never
 *   throws across the ABI.  gpw_last_error() gives a message for the calling thread.
 */
#ifndef GPW_H_
#define GPW_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GPW_OK 0
#define GPW_EINVAL -1     /* bad argument: l > 3, degenerate lattice, bad mesh, NULL */
#define GPW_ENOMEM -2     /* device or host allocation failed */
#define GPW_ECUDA -3      /* CUDA runtime error */
#define GPW_ECUFFT -4     /* cuFFT error */
#define GPW_ETIMEDOUT -5  /* a bounded wait gave up (gpw_stream_wait) */
#define GPW_EDEVICE -6    /* a kernel's bounds check set the device error word */
#define GPW_ERANGE -7     /* a size is beyond a fixed limit of the library */

#define GPW_MAX_LEVELS 8

/* Flags for gpw_desc.flags */
#define GPW_STRICT 0            /* default: the truncation definition of the paper */
#define GPW_TAU 1               /* also build the kinetic-energy-density (meta-GGA) data:
                                   1-D tables to degree L+3 and larger per-pair buffers;
                                   shells up to f (gpw_eval_tau, gpw_eval_mat_tau*) */
#define GPW_HOST_TASKS 2        /* build the sub-box task records and work lists on the
                                   host in gpw_plan_prepare.  Default: the host only
                                   counts each pair's tasks and gpw_plan_commit builds
                                   the records on the device (count per grid block,
                                   prefix sums, fill: the pair-to-block mapping of the
                                   paper's appendix); both give identical lists. */
#define GPW_FAST_BLOCK_PRUNE 4  /* per-block value screening (App. Alg. 5): drop from the
                                   collocation task lists every (pair, sub-box) task whose
                                   part of the pair box lies wholly farther than R_p from
                                   the pair centre P (every point there has its Eq. cut
                                   bound below tau).  Which points are dropped depends on
                                   the sub-box shape, so this is outside the strict
                                   definition: densities and energies move by tau-sized
                                   amounts (checked at 1e-6 relative).  Integration keeps
                                   every task.  Orthorhombic cells use the distance to the
                                   task's box; non-orthogonal cells two lower bounds of it
                                   (the largest distance across the lattice-plane slabs,
                                   and the fractional distance times the square root of the
                                   lattice metric's smallest eigenvalue). */
#define GPW_DEBUG_CHECKS 8      /* extra device checks, read with gpw_check_device: at
                                   commit every task record of both lists is checked
                                   against its sub-box and its pair's box (code 17), and
                                   every evaluation checks its outputs (V, gradient,
                                   energies, densities) for values that are not finite
                                   (code 16).  Results are unchanged. */

/* Exchange functional (gpw_desc.xc), spin-unpolarised, on the finest grid:
 * GPW_XC_LDA_X  Slater exchange v_x = -(3/pi)^(1/3) rho^(1/3) (Sec. II, LDA);
 * GPW_XC_PBE_X  PBE exchange, a GGA (Sec. II, GGA): grad rho = F^-1(i G rho~(G)),
 *               e = e_x^LDA(rho) F_x(s), F_x = 1 + kappa - kappa/(1 + mu s^2/kappa),
 *               s = |grad rho| / (2 (3 pi^2)^(1/3) rho^(4/3)), kappa = 0.804,
 *               mu = 0.21951; the potential de/drho - div(de/d grad rho) with the
 *               divergence as F^-1(i G . F(.)) (the integration by parts that folds the
 *               GGA term into the local potential).  Derivatives take the Nyquist plane
 *               of an even mesh axis as zero; e = 0 where rho <= 1e-12. */
#define GPW_XC_LDA_X 0
#define GPW_XC_PBE_X 1

typedef struct gpw_plan_s* gpw_plan_t;
typedef struct gpw_batch_s* gpw_batch_t;

/* Problem statement (Sec. II and III A of the paper): cell, atoms, Gaussian shells,
 * plane-wave cutoff and multigrid levels, screening threshold tau of Eq. (cut).
 * All pointers are host memory, read during gpw_plan only. */
typedef struct {
  double lattice[9];          /* rows a1, a2, a3 (Bohr), linearly independent; a
                                 non-diagonal lattice is a non-orthogonal cell: images
                                 T = n . rows, boxes from the reciprocal rows, meshes
                                 from the row lengths |a_d| */
  int natm;
  const double* coords;       /* natm x 3 atom positions (Bohr) */
  int nshell;
  const int* shell_atom;      /* nshell: atom of each shell */
  const int* shell_l;         /* nshell: angular momentum 0..3 */
  const int* shell_nprim;     /* nshell: primitives in the shell */
  const int* shell_prim_off;  /* nshell: first primitive in exponents/coeffs */
  const double* exponents;    /* primitive exponents alpha (Bohr^-2) */
  const double* coeffs;       /* contraction coefficients (unnormalised; each primitive
                                 is multiplied by N_l(alpha), unit x^l self-overlap) */
  double cutoff_ha;           /* finest-level cutoff E_0 (Hartree); ignored if meshes */
  int nlevels;                /* 1..GPW_MAX_LEVELS */
  double level_ratio;         /* E_k = E_0 / ratio^k */
  const int* meshes;          /* optional nlevels x 3 explicit meshes; NULL = derive */
  double rel_cutoff;          /* a pair of exponent alpha_p goes to the coarsest level
                                 with E_k >= rel_cutoff * alpha_p (40 if <= 0) */
  double tau;                 /* screening threshold of Eq. (cut) */
  int flags;                  /* GPW_STRICT, or GPW_TAU | GPW_HOST_TASKS |
                                 GPW_FAST_BLOCK_PRUNE | GPW_DEBUG_CHECKS */
  int tile[3];                /* sub-box owned by one collocation thread block (grid
                                 points along a1, a2, a3); {0,0,0} = default {4,8,16} */
  int tile_integ[3];          /* sub-boxes of the integration (grid points along a1, a2,
                                 a3; along a3 the stride of the z windows, see
                                 integ_zwin); {0,0,0} = the default: {8,8,16} with
                                 48-point z windows where the staging of the plan's
                                 largest degree leaves two thread blocks per SM, else
                                 {8,8,32}; non-orthogonal cells {4,8,16}.  Supported
                                 shapes: gpw_tile_supported, gpw_integ_zwin_supported. */
  int colloc_warps;           /* warps per collocation thread block: 4, 6 or 8; 0 = the
                                 choice with the most resident warps per SM (the
                                 larger block on a tie) */
  int integ_chunk;            /* most (pair, sub-box) tasks per integration work item
                                 (> 0); 0 = default max(64, tasks / 1216) */
  int xc;                     /* GPW_XC_LDA_X (0, default) or GPW_XC_PBE_X */
  int host_threads;           /* most host threads the planner uses (>= 0); 0 = OpenMP's
                                 default (all cores).  A server planning several cells
                                 at once on its own threads caps each plan here. */
  int integ_zwin;             /* z extent (grid points) of the window one integration
                                 thread block stages: a multiple of tile_integ[2], whose
                                 sub-boxes then overlap along a3.  A pair box is cut
                                 along a3 where a window starting in its current
                                 sub-box ends, not at every sub-box boundary, so a
                                 task's first (z) contraction runs over up to zwin
                                 points and its y contraction once per window instead
                                 of once per sub-box (the V tensor of Sec. III A; the
                                 sums are the same, in another order).  0 = the
                                 default: tile_integ[2] when tile_integ is given, else
                                 what the default sub-boxes take; a non-zero value
                                 needs an explicit tile_integ (GPW_EINVAL otherwise,
                                 and for shapes gpw_integ_zwin_supported rejects). */
} gpw_desc;

/* Sizes and work counts of a plan (gpw_plan_query). */
typedef struct {
  int nao, natm, nlevels, lmax;
  int meshes[GPW_MAX_LEVELS][3];
  double level_cutoff[GPW_MAX_LEVELS];  /* E_k (Hartree) */
  long long npairs;
  long long npairs_level[GPW_MAX_LEVELS];
  long long pair_points;                 /* sum over pairs of box volumes */
  long long pair_points_level[GPW_MAX_LEVELS];
  long long pair_points_L[8];            /* by la + lb */
  long long nentries;                    /* (pair, sub-box) collocation tasks (those kept,
                                            once committed with GPW_FAST_BLOCK_PRUNE) */
  long long device_bytes;                /* device memory owned by the plan */
  double flops_rho;    /* model FP64 flops of one eval_rho grid pass: 2 (L+1) per pair-point */
  double flops_mat;    /* same for eval_mat */
  double flops_ip1;    /* 2 (L+2) per pair-point for eval_mat_ip1 */
  int tile[3];         /* collocation sub-box */
  int tile_integ[3];   /* integration sub-box */
  long long nentries_integ;  /* tasks of the integration sub-box lists */
  int colloc_warps;    /* warps per collocation block (0 until the plan is committed) */
  int integ_chunk;     /* most tasks per integration work item */
  int xc;              /* exchange functional (GPW_XC_*) */
  double volume;       /* cell volume Omega = |det(lattice)| (Bohr^3) */
  double weight[GPW_MAX_LEVELS];  /* grid weight Omega / N_k of level k: the quadrature
                                     weight of eval_mat, the gradient and the energies */
  int integ_zwin;      /* z window of the integration sub-boxes (= tile_integ[2]: plain
                          tiling) */
} gpw_plan_info;

/* Build a plan: normalise primitives, screen pairs (Eq. cut; pairs a <= b over images T
 * with |A - B - T| < r_a + r_b, Sec. III A), assign levels, build the per-level
 * sub-box task lists, allocate grids/spectra/cuFFT plans, and precompute the 1-D
 * Gaussian factor tables of Eq. (gab_lp) on the device (enqueued on `stream`).
 * On a non-orthogonal cell the 1-D tables hold the diagonal part of the Gaussian in
 * grid units along the rows, the grid kernels multiply in the cross factors
 * exp(-2 alpha_p G_de eta_d eta_e) (the row-to-row terms of the appendix recursion), and
 * pair tensors are re-expanded between Cartesian and row monomials.
 * Returns GPW_EINVAL for a degenerate lattice, l > 3, nlevels outside
 * 1..GPW_MAX_LEVELS, non-positive exponents, meshes too small for the cutoff sphere,
 * or other sub-boxes on a non-orthogonal cell.  *out is set only on success. */
int gpw_plan(const gpw_desc* desc, void* stream, gpw_plan_t* out);

/* Host phase of gpw_plan only: screening, levels and task lists on the CPU, no device
 * work and no device allocation.  gpw_plan_query then reports the exact device_bytes
 * the commit will allocate (cuFFT work areas estimated), which lets a scheduler admit
 * the plan by device memory before committing it.  Evaluations need a committed plan. */
int gpw_plan_prepare(const gpw_desc* desc, gpw_plan_t* out);

/* Device phase: allocate and upload the plan, create cuFFT plans and the 1-D tables
 * (enqueued on `stream`).  On failure the plan stays prepared and can be retried. */
int gpw_plan_commit(gpw_plan_t plan, void* stream);

/* Which kernels exist for the sub-box shape (t0, t1, t2): a mask of GPW_TILE_COLLOC
 * (usable as gpw_desc.tile) and GPW_TILE_INTEG (usable as gpw_desc.tile_integ); 0 if
 * neither. */
#define GPW_TILE_COLLOC 1
#define GPW_TILE_INTEG 2
int gpw_tile_supported(int t0, int t1, int t2);

/* 1 if an integration kernel exists for sub-boxes (t0, t1, t2) whose thread blocks stage
 * z windows of zwin grid points (gpw_desc.integ_zwin; zwin = t2 for every shape that
 * gpw_tile_supported marks GPW_TILE_INTEG), else 0. */
int gpw_integ_zwin_supported(int t0, int t1, int t2, int zwin);

/* Fill *info (host). */
int gpw_plan_query(gpw_plan_t plan, gpw_plan_info* info);

/* Move the atoms to `coords` (host, natm x 3) keeping the pair set, images, levels
 * and integer boxes of the plan frozen (the energy is then smooth in the coordinates,
 * which is what finite differences of the gradient need).  Recomputes the tables. */
int gpw_plan_update_coords(gpw_plan_t plan, const double* coords, void* stream);

/* Copy the screened pair table to host arrays of plan.npairs rows (any may be NULL):
 * ab (2 ints: primitive indices a <= b), img (3 ints n: the image T = sum_d n_d R_d of b
 * over the lattice rows R_d, n . diag(L) for an orthorhombic cell), level, lo/hi (3 ints
 * each: integer box on the level mesh along the rows, inclusive).  Synchronous. */
int gpw_plan_pairs(gpw_plan_t plan, int* ab, int* img, int* level, int* lo, int* hi);

/* Copy one task list of a committed plan to host buffers (any may be NULL): integ = 0
 * the collocation list, 1 the integration list.  *nent tasks (8 ints each: the two int4
 * records p, m | L << 24, u, rank and t0, t1, t2, W offset), *nsub + 1 sub-box CSR
 * offsets, *nwork work items (4 ints: plan slot, level | chunk << 4, sub-box, tasks).
 * The counts are written first, so a call with NULL buffers sizes them.  With
 * GPW_FAST_BLOCK_PRUNE the collocation list holds the tasks kept (their rank field still
 * numbers all of the pair's tasks).  Synchronises the device. */
int gpw_plan_task_lists(gpw_plan_t plan, int integ, long long* nent, long long* nsub,
                        long long* nwork, int* tasks, long long* sub_off, int* work);

/* Density on the finest grid (Eq. rho_wrap + multigrid Fourier interpolation).
 * D: device, nao x nao symmetric.  rho_fine: device, N0*N1*N2 of level 0 (overwritten). */
int gpw_eval_rho(gpw_plan_t plan, const double* D, double* rho_fine, void* stream);

/* Raw per-level densities before interpolation: rho_levels[k] (device, N_k doubles,
 * overwritten) for k < nlevels (an entry may be NULL to skip copying that level). */
int gpw_eval_rho_levels(gpw_plan_t plan, const double* D, double* const* rho_levels,
                        void* stream);

/* V_mu,nu = sum_k sum_pairs (Omega/N_k) sum_r v_k(r) phi_mu phi_nu (Eq. J_wrap), where
 * v_k is v_fine restricted to level k (keep |G| < G_k).  v_fine: device, finest grid.
 * V: device nao x nao, overwritten (symmetric). */
int gpw_eval_mat(gpw_plan_t plan, const double* v_fine, double* V, void* stream);

/* As gpw_eval_mat with the level potentials given directly (device pointers,
 * N_k doubles each); no restriction is applied. */
int gpw_eval_mat_levels(gpw_plan_t plan, const double* const* v_levels, double* V,
                        void* stream);

/* Hxc nuclear gradient dE/dR = <v_Hxc, d rho / dR> (Algorithm 3) for the density
 * matrix D (device) and the finest-grid potential v_fine (device), with the boxes of
 * the plan held fixed.  grad: device natm x 3, overwritten. */
int gpw_eval_mat_ip1(gpw_plan_t plan, const double* D, const double* v_fine, double* grad,
                     void* stream);

/* As gpw_eval_mat_ip1 with per-level potentials (device, N_k doubles each). */
int gpw_eval_mat_ip1_levels(gpw_plan_t plan, const double* D, const double* const* v_levels,
                            double* grad, void* stream);

/* Kinetic energy density of meta-GGA functionals (Sec. II, meta-GGA; Eq. J_metaGGA and
 * the tau terms of Algorithms 2 and 3): tau(r) = (1/2) sum D_mu,nu grad phi_mu . grad phi_nu
 * collocated on the pairs' levels like rho and Fourier-interpolated to the finest grid,
 * its Fock term V_mu,nu = (1/2) sum_k sum_pairs (Omega/N_k) sum_r v_k grad phi_mu . grad phi_nu
 * and the nuclear gradient of <v, tau(D)> at fixed v.  Need a plan built with GPW_TAU
 * (shells up to f: the pair tensors reach degree L + 2 = 8 and, for the gradient,
 * L + 3 = 9); GPW_EINVAL otherwise.  Arguments as for the rho / V / gradient calls
 * above (device pointers; outputs overwritten). */
int gpw_eval_tau(gpw_plan_t plan, const double* D, double* tau_fine, void* stream);
int gpw_eval_tau_levels(gpw_plan_t plan, const double* D, double* const* tau_levels,
                        void* stream);
int gpw_eval_mat_tau(gpw_plan_t plan, const double* v_fine, double* V, void* stream);
int gpw_eval_mat_tau_levels(gpw_plan_t plan, const double* const* v_levels, double* V,
                            void* stream);
int gpw_eval_mat_tau_ip1(gpw_plan_t plan, const double* D, const double* v_fine, double* grad,
                         void* stream);
int gpw_eval_mat_tau_ip1_levels(gpw_plan_t plan, const double* D,
                                const double* const* v_levels, double* grad, void* stream);

/* One Fock build: rho = eval_rho(D); v_H from Eqs. (vH)/(vHG) with G = 0 dropped;
 * Slater exchange v_x = -(3/pi)^(1/3) max(rho,0)^(1/3); v = v_H + v_x restricted to
 * every level; V = eval_mat.  energies (host, 2 doubles): E_H = (1/2)<rho, v_H> and
 * E_x = (Omega/N) sum e_x; the call synchronises `stream` to return them.
 * rho_out and v_fine_out (device, finest grid) are optional (NULL). */
int gpw_fock(gpw_plan_t plan, const double* D, double* V, double* energies,
             double* rho_out, double* v_fine_out, void* stream);

/* As gpw_fock without the final synchronisation: the two energies are written to
 * `energies_dev` (device, 2 doubles) on `stream`.  Usable inside CUDA-graph capture. */
int gpw_fock_async(gpw_plan_t plan, const double* D, double* V, double* energies_dev,
                   double* rho_out, double* v_fine_out, void* stream);

/* Fock build plus Hxc gradient in one pass: the level potentials of the build are
 * integrated once at degree L + 1 per pair, which yields both V (Algorithm 2) and the
 * gradient contraction (Algorithm 3) with the density matrix D.  V (device nao x nao),
 * grad (device natm x 3), energies (host, 2 doubles; the call synchronises `stream`). */
int gpw_fock_grad(gpw_plan_t plan, const double* D, double* V, double* grad, double* energies,
                  void* stream);

/* gpw_fock_grad from and to HOST memory: D (host nao x nao) is copied to the device, the
 * Fock build and gradient run on `stream`, and V (host nao x nao), grad (host natm x 3)
 * and energies (host, 2 doubles) are copied back; returns after synchronising `stream`
 * and the plan's own copy stream, which takes V back while the gradient kernels run.
 * Pinned (page-locked) host buffers give full-rate copies; pageable ones work too.  The
 * first call on a plan allocates the plan's device copies of D, V and the gradient
 * (2 nao^2 + 3 natm doubles) and creates that stream and one event, all kept until the
 * plan is destroyed; later calls allocate nothing.  Not a paper operation: the
 * end-to-end form of the same build. */
int gpw_fock_grad_host(gpw_plan_t plan, const double* D, double* V, double* grad,
                       double* energies, void* stream);

/* As gpw_fock_grad with the energies written to device memory (2 doubles), no sync. */
int gpw_fock_grad_async(gpw_plan_t plan, const double* D, double* V, double* grad,
                        double* energies_dev, void* stream);

/* Batches: the collocation and integration tasks of several plans (cells) run in one
 * launch each, instead of one launch per plan: every plan's work list is cut into runs
 * of consecutive items (neighbouring sub-boxes) and the runs of all plans go by
 * decreasing mean weight.  The other steps run per plan on the same stream.  Plans of a batch share their
 * sub-box shapes and device.  Results per plan are identical to the plan run alone (the
 * same tasks, in the same order per sub-box, with the same reductions). */
int gpw_batch_create(int max_plans, gpw_batch_t* out);

/* Attach nplans committed plans (<= max_plans): builds the merged work lists and the
 * device views (synchronises `stream`).  Call again whenever the plan set changes. */
int gpw_batch_set(gpw_batch_t batch, int nplans, const gpw_plan_t* plans, void* stream);

/* gpw_fock_grad_async for every attached plan i: D[i], V[i] device nao_i x nao_i,
 * grad[i] device natm_i x 3 (grad or grad[i] may be NULL to skip the gradient),
 * energies_dev device 2*nplans doubles (E_H, E_x of plan i at 2i, 2i+1).  Allocates
 * nothing and does not synchronise, so the sequence can be captured in a CUDA graph.
 * A captured graph holds the plan set, launch shapes and device work lists in force at
 * capture: every later gpw_batch_set (which may free and refill those lists) makes it
 * invalid, and it must not be replayed after one.  Capture again when
 * gpw_batch_generation has changed; destroying a plan of the set also invalidates it. */
int gpw_batch_fock_grad_async(gpw_batch_t batch, const double* const* D, double* const* V,
                              double* const* grad, double* energies_dev, void* stream);

/* Number of successful gpw_batch_set calls on the batch so far (0 after create): a graph
 * captured at generation g is valid only while the generation is still g.  Not a paper
 * operation. */
int gpw_batch_generation(gpw_batch_t batch, long long* generation);

void gpw_batch_destroy(gpw_batch_t batch);

/* Read and clear the device error word of the plan (synchronises `stream`).
 * Returns GPW_OK, or GPW_EDEVICE with *code set to the first recorded check: 1 a
 * collocation task record outside its sub-box or its pair's tables, or a pair degree
 * beyond the compiled collocation bodies (the task, or the pair's contracted table, is
 * skipped), 3 the same for integration, 16 a value that is not finite in an output and
 * 17 an inconsistent task list at commit (both with GPW_DEBUG_CHECKS). */
int gpw_check_device(gpw_plan_t plan, int* code, void* stream);

/* Phases timed by the profiler (gpw_profile). */
#define GPW_PHASE_COEF 0            /* pair D tensors (Eq. rho1) and their x contraction */
#define GPW_PHASE_COLLOCATE 1       /* collocation kernel (Algorithm 1) */
#define GPW_PHASE_SPECTRAL 2        /* FFTs, interpolation, Poisson, exchange, restriction */
#define GPW_PHASE_INTEGRATE 3       /* integration kernel (Algorithm 2) */
#define GPW_PHASE_ASSEMBLE 4        /* per-pair reductions and V assembly */
#define GPW_PHASE_INTEGRATE_IP1 5   /* integration kernel at degree L+1 (Algorithm 3) */
#define GPW_PHASE_GRAD 6            /* gradient contraction and per-atom sums */
#define GPW_NPHASES 7

/* Device timing of later calls on this plan, per phase, with CUDA events recorded on
 * each call's stream.  enable != 0 clears the totals and starts recording; 0 stops.
 * Not for use inside CUDA-graph capture. */
int gpw_profile(gpw_plan_t plan, int enable);

/* Synchronise the recorded events and return, per phase (up to nphases entries),
 * the summed milliseconds (ms) and the number of timed intervals (count); either
 * pointer may be NULL.  *launches (optional) receives the number of libgpw kernels
 * launched on this plan since the plan was built (cuFFT's own kernels excluded). */
int gpw_profile_read(gpw_plan_t plan, double* ms, long long* count, int nphases,
                     long long* launches);

/* Largest density grid gpw_lda_x_noalloc accepts (points). */
#define GPW_LDA_NOALLOC_MAX_POINTS 67108864

/* Slater exchange of a density grid without any device allocation and without a plan.
 * The paper has no counterpart to this entry point: it exists for callers that cannot
 * call cudaMalloc (an application whose memory pool owns the device, a loop that must
 * not enter the driver's allocator, a library that does not own the CUDA context).
 * rho: device, n doubles (n <= GPW_LDA_NOALLOC_MAX_POINTS, else GPW_ERANGE);
 * v_x: device, n doubles, overwritten with -(3/pi)^(1/3) max(rho,0)^(1/3);
 * e_x: device, 1 double, overwritten with weight * sum -(3/4)(3/pi)^(1/3) max(rho,0)^(4/3)
 *      (weight = Omega / n gives E_x of gpw_fock).
 * The working memory is one fixed 32 KB array in the library's device image, shared by
 * every call on a GPU and keeping the last call's contents (each call writes what it
 * reads, so nothing needs clearing); calls whose executions overlap on the GPU race on
 * it.  The first call in each CUDA context (normally once per device) looks up the
 * array's device address, and with lazy module loading (CUDA's default) that lookup loads
 * the library's device image onto the device, which may allocate inside the driver: make
 * that first call during set-up, with the device current and before any stream capture.
 * Later calls in the same context reuse the address; a context created later (after a
 * device reset, or another context on the device) has its own first call.
 * Asynchronous on `stream`. */
int gpw_lda_x_noalloc(const double* rho, long long n, double weight, double* v_x, double* e_x,
                      void* stream);

/* Bounded host wait: returns GPW_OK once every piece of work enqueued on `stream` so far
 * has finished, or GPW_ETIMEDOUT when that has not happened within timeout_s seconds
 * (>= 0; the work is not cancelled and keeps running).  Polls cudaStreamQuery with short
 * sleeps, so the calling thread does not spin a core.  GPW_ECUDA if the stream reports
 * an error.  Not a paper operation: a server uses it to put a deadline on a batch. */
int gpw_stream_wait(void* stream, double timeout_s);

/* Release the plan and everything it owns.  NULL is ignored. */
void gpw_plan_destroy(gpw_plan_t plan);

/* As gpw_plan_destroy, without synchronising the device: the plan's memory returns to
 * the device pool in stream order on `stream`.  The caller guarantees that every piece of
 * work that uses the plan has finished or is ordered before `stream` (a server that
 * waited for a request's batch).  Not a paper operation. */
void gpw_plan_destroy_async(gpw_plan_t plan, void* stream);

/* Static message for an error code. */
const char* gpw_strerror(int code);

/* Message of the last failing call on this thread ("" if none). */
const char* gpw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GPW_H_ */
