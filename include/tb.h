/*
 * tb.h - C ABI of the GB300 linear-scaling tight-binding force library.
 *
 * The library evaluates, for every target atom of a periodic cubic cell, the
 * local electronic structure of the paper's linear-scaling method:
 *   cluster of atoms within the cutoff radius (Sec. 2, locality),
 *   block Krylov space seeded with the target's four sp3 orbitals
 *   (Sec. 3, Eq. (Krylov), block form of Eqs. (lanczos)/(lanczos_blas3)),
 *   eigenpairs of the projected matrix T = V^T H V (Sec. 3),
 *   density-matrix columns rho|i,a> with the occupation f(e) (Sec. 2),
 *   a global chemical potential, and forces <F_i> = Tr[rho F_i] (Sec. 2),
 * on the Hamiltonian of Eq. (1) (orthogonal sp3 Slater-Koster model with GSP
 * distance scaling; Sec. 5 names Xu's parameterisation and its 2.6 A cutoff).
 *
 * General rules
 *  - Every array argument is a DEVICE pointer owned by the caller, unless the
 *    argument's comment says "host".  The library owns only the opaque context
 *    (parameters, device workspace, a device status word).
 *  - Every call is ordered on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream) and returns without synchronising the host.
 *    After tb_ctx_reserve no call allocates memory, so the call sequence can be
 *    captured into a CUDA graph.  tb_ctx_create / tb_ctx_reserve /
 *    tb_ctx_destroy / tb_get_status are not capturable.
 *  - Host-side argument errors return a status at once.  Problems detected on
 *    the device (capacity overflow, non-finite values, eigen-iteration or mu
 *    non-convergence, a wait that timed out, positions outside [0, L)) are
 *    written to the context's device status word (first error wins) and are
 *    read back with tb_get_status.  No call traps or aborts.
 *  - Units: A, eV, fs, amu.  Forces in eV/A.  Positions must lie in [0, L).
 *  - Orbital order on every atom: s, px, py, pz.
 *  - Index type int32; sizes are int.
 */
#ifndef TB_H
#define TB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tb_status {
  TB_OK = 0,
  TB_ERR_INVALID_ARG = 1,     /* bad pointer/size/parameter, or position outside [0,L) */
  TB_ERR_CUDA = 2,            /* a CUDA runtime call failed                            */
  TB_ERR_NOMEM = 3,           /* workspace allocation failed (tb_ctx_reserve only)     */
  TB_ERR_CAPACITY = 4,        /* a list or cluster exceeded max_hnbr / max_cluster     */
  TB_ERR_NONFINITE = 5,       /* NaN/Inf met in an input or intermediate              */
  TB_ERR_BREAKDOWN = 6,       /* Krylov seed block lost rank (cannot happen for E_i)   */
  TB_ERR_NO_CONVERGENCE = 7,  /* projected eigensolve or mu search did not converge    */
  TB_ERR_TIMEOUT = 8,         /* a bounded device-side wait gave up                    */
  TB_ERR_NOT_RESERVED = 9     /* workspace missing or too small for n                  */
} tb_status;

typedef enum tb_precision {
  /* Everything in FP64. */
  TB_PREC_FP64 = 0,
  /* H.V sweeps, Krylov basis and its inner products, and the projected
   * eigensolve in FP32; the block tridiagonal T in FP64, eigenvalues as
   * Rayleigh quotients on T in double-float arithmetic; mu (FP64 Newton, FP32
   * terms for pairs far from mu), density-matrix blocks, energies and forces
   * in FP64. */
  TB_PREC_MIXED = 1,
  /* As TB_PREC_MIXED, with the H.V sweeps in BF16: the Slater-Koster records
   * and the Krylov block V_k enter the sweep's products rounded to BF16
   * (8-bit mantissa), the products accumulated in FP32.  Not available with
   * the m-target form (group_m > 1). */
  TB_PREC_BF16 = 2
} tb_precision;

/* Model and numerical parameters (all lengths A, energies eV). */
typedef struct tb_params {
  /* Eq. (1): on-site energies and Slater-Koster two-centre integrals at r0 */
  double Es, Ep, Vss, Vsp, Vpps, Vppp;
  /* hopping scaling s(r) = (r0/r)^n exp{n[-(r/rc)^nc + (r0/rc)^nc]} */
  double r0, n, nc, rc;
  /* pair repulsion phi(r) = phi0 (d0/r)^m exp{m[-(r/dc)^mc + (d0/dc)^mc]} */
  double phi0, d0, m, mc, dc;
  /* C1 cubic tail on [r1, rm]; s and phi vanish for r >= rm (the hopping
   * cutoff; the Hamiltonian neighbour list uses r <= rm) */
  double r1, rm;
  double kT;          /* Fermi smearing (eV), > 0                                */
  double Rc;          /* cluster cutoff radius (A), Rc >= rm, Rc < L/2 advisable */
  double defl_tol;    /* absolute deflation threshold on a new Krylov column (eV)*/
  double mu_tol;      /* mu search stops when |N(mu) - N_e| <= mu_tol * N_e      */
  int r;              /* Krylov block order: basis of r blocks, 4r columns, 1..16 */
  int prec;           /* tb_precision                                            */
  int max_hnbr;       /* capacity of one Hamiltonian neighbour list, <= 256      */
  int max_cluster;    /* capacity of one cluster (target included), <= 1024      */
  int reorth_passes;  /* classical Gram-Schmidt passes against all blocks: 1 or 2*/
  int mu_max_iter;    /* cap on mu search passes (e.g. 100)                      */
  long long timeout_cycles; /* budget of any device spin-wait, in SM clocks      */
  int reorth_every;   /* full reorthogonalisation against all earlier blocks
                       * every this many Lanczos steps (>= 1; 1 = every step);
                       * the other steps project out the last two blocks only */
  int group_m;        /* targets per group of the m-target form (1..4; 1 = one
                       * target per cluster, the default); see tb_group_atoms */
  int max_union;      /* capacity of a group's union cluster (atoms, <= 1024);
                       * 0 = min(1024, group_m * max_cluster)                   */
  int schedule;       /* tb_schedule: how the mixed path's block Lanczos and
                       * projected eigensolve are launched                      */
} tb_params;

typedef enum tb_schedule {
  /* The library chooses: its own measurement when tb_autotune has run on
   * this context, else the persistent queue when the targets fill at most 16
   * waves of CTAs and separate launches otherwise. */
  TB_SCHED_AUTO = 0,
  /* One persistent launch: a work queue of block-Lanczos targets followed by
   * projected-eigensolve items, so the eigensolves fill the SMs the last
   * Krylov targets leave idle (mixed path, single-target clusters). */
  TB_SCHED_PERSISTENT = 1,
  /* Separate block-Lanczos and eigensolver launches. */
  TB_SCHED_SEPARATE = 2,
  /* The persistent queue with the targets taken in decreasing cluster size
   * (the longest block-Lanczos runs start first; one more small launch sorts
   * the targets into size bins of 8 atoms). */
  TB_SCHED_PERSISTENT_LARGEST_FIRST = 3,
  /* Separate launches per cluster-size bucket, each with its own tile: the
   * bucket's largest cluster sizes the shared-memory basis blocks, with its
   * own share of shared memory for the Slater-Koster records and its own
   * register budget (CTAs per SM); then the eigensolver.  Buckets and tiles
   * come from tb_autotune, else four equal size ranges up to max_cluster. */
  TB_SCHED_BUCKETED = 4
} tb_schedule;

typedef struct tb_ctx tb_ctx;

/* Fill *p with the library defaults for numerical fields (model constants are
 * zeroed: the caller sets them).  Host pointer.  Never fails for p != NULL. */
tb_status tb_params_default(tb_params* p);

/* Create a context on the current CUDA device.  *out (host) receives the
 * handle.  Validates *p (host).  Allocates a small device status word.  */
tb_status tb_ctx_create(tb_ctx** out, const tb_params* p);

/* Free the context and its workspace.  Synchronises the device. */
tb_status tb_ctx_destroy(tb_ctx* ctx);

/* Allocate (or grow) the device workspace for systems of up to n_atoms atoms.
 * The only call after tb_ctx_create that allocates.  Synchronises. */
tb_status tb_ctx_reserve(tb_ctx* ctx, int n_atoms);

/* Bytes of device workspace currently held (host out). */
tb_status tb_ctx_workspace_bytes(const tb_ctx* ctx, size_t* bytes);

/* Read and clear the device status word: *code (host) gets a tb_status, *info
 * (host) an index or size qualifying it (e.g. the offending atom or the
 * capacity that would have been needed).  Synchronises `stream`. */
tb_status tb_get_status(tb_ctx* ctx, int* code, int* info, void* stream);

/*
 * Neighbour and cluster lists (Sec. 2: atoms within the cutoff radius of
 * the target).  Candidates come from cell lists (cells of side >= Rc + 0.01 A)
 * when the box holds at least 3 such cells per dimension, else from all
 * pairs; an FP32 prefilter drops far pairs, and the membership decision is the
 * FP64 test below, so the lists are bit-exact and the same on both paths:
 *   d = x_j - x_i;  d -= L if d > L/2;  d += L if d < -L/2   (per component)
 *   r2 = (dx*dx + dy*dy) + dz*dz   (each operation rounded, no FMA)
 *   Hamiltonian list of i: all j != i with r2 <= rm*rm, ascending j;
 *   cluster of i: i itself first, then all j != i with r2 <= Rc*Rc, ascending.
 * pos   [n*3]  FP64, row-major (x,y,z per atom), each in [0, L)
 * h_off [n+1]  out, CSR offsets of the Hamiltonian lists
 * h_idx [n*max_hnbr] out (capacity), CSR column indices
 * c_off [n+1]  out, CSR offsets of the clusters
 * c_idx [n*max_cluster] out (capacity)
 * A list longer than its capacity sets TB_ERR_CAPACITY (info = the length
 * needed) and is truncated to the capacity.
 */
tb_status tb_build_neighbors(tb_ctx* ctx, int n, const double* pos, double L,
                             int* h_off, int* h_idx, int* c_off, int* c_idx,
                             void* stream);

/*
 * Hamiltonian blocks of Eq. (1) for every directed bond p = (i -> j),
 * j = h_idx[p], d = R_j - R_i (minimum image), l = d/|d|:
 *   Hblk[p*16 + a*4 + b]      = H_{i a, j b} = s(|d|) * SK_ab(l)
 *   dHblk[p*48 + k*16 + a*4 + b] = d H_{i a, j b} / d d_k
 *   (so dH/dR_i = -dHblk and dH/dR_j = +dHblk).
 * The on-site block diag(Es, Ep, Ep, Ep) is implicit (not stored).
 * Hsk (may be NULL for TB_PREC_FP64, required otherwise): the FP32
 * Slater-Koster record of each directed bond, [p*4 + 0..3] =
 * (s(|d|), l_x, l_y, l_z), from which the block is s(|d|) SK(l) with the
 * context's Vss, Vsp, Vpps, Vppp; the mixed and BF16 paths sweep with these
 * 16-byte records instead of the 128-byte FP64 blocks.  Arrays sized by
 * h_off[n] entries.
 */
tb_status tb_assemble_H(tb_ctx* ctx, int n, const double* pos, double L,
                        const int* h_off, const int* h_idx,
                        double* Hblk, double* dHblk, float* Hsk,
                        void* stream);

/*
 * Per target atom i: cluster map, block Krylov space of order r from
 * V_1 = E_i (the four orbitals of i), block Lanczos with full
 * reorthogonalisation and deflation, T = block tridiagonal (A_k, B_k), its
 * eigenpairs (lam_m, U), and the spectral record.  With NT = 4r and kdim[i]
 * the number of Krylov columns kept (<= NT):
 *   lambda[i*NT + m]            Ritz values, ascending, m < kdim[i]; 0 beyond
 *   S[(i*4 + a)*NT + m]          = U[a][m], the seed-block components
 *   P[((i + h_off[i] + q)*4 + b)*NT + m] = sum_l V[row(q,b)][l] U[l][m]
 *       q = 0 is the target itself, q = 1..deg(i) its Hamiltonian neighbours
 *       in h_idx order; P needs (n + h_off[n]) * 4 * NT doubles
 *   kdim[i]                      int
 * Then rho_{(q) b, i a} = sum_m P[q,b,m] f((lam_m - mu)/kT) S[a,m].
 * TB_PREC_FP64 sweeps with Hblk; the other precisions with the records Hsk
 * of tb_assemble_H (must be non-NULL), staged in shared memory per target.
 */
tb_status tb_krylov_density(tb_ctx* ctx, int n, const int* c_off, const int* c_idx,
                            const int* h_off, const int* h_idx,
                            const double* Hblk, const float* Hsk,
                            double* lambda, double* S, double* P, int* kdim,
                            void* stream);

/*
 * Chemical potential: solves 2 sum_i sum_m w_im f((lam_im - mu)/kT) = N_e
 * with w_im = sum_a S[i,a,m]^2 and f(x) = 1/(1+e^x), by bracketed Newton
 * steps with bisection fallback, in FP64, in one cooperative launch.
 * mu_guess (device, may be NULL): starting point if inside the bracket.
 * mu (device, out): one double.  n_count (device, out, may be NULL): N(mu).
 * Stops when |N(mu) - N_e| <= mu_tol * N_e or the bracket is below 1e-13 eV,
 * or after a Newton step whose residual is bounded by a tenth of that
 * tolerance (|N''| <= N'/kT bounds it by r^2 / (2 kT N') from the previous
 * residual r); then n_count is that step's predicted count, N_e.  After
 * mu_max_iter passes sets TB_ERR_NO_CONVERGENCE (mu = best estimate).
 */
tb_status tb_find_mu(tb_ctx* ctx, int n, const double* lambda, const double* S,
                     const int* kdim, double n_electrons, const double* mu_guess,
                     double* mu, double* n_count, void* stream);

/*
 * Density-matrix blocks, energies and forces (Sec. 2: <F> = Tr[rho F]).
 *   rho^(i)_{q b, i a} = sum_m P[q,b,m] f_m S[a,m]
 *   F_k = 2 sum_{j in H(k)} sum_{a,b} [rho^(k)_{j b,k a} + rho^(j)_{k a,j b}]
 *         dHblk(k->j)_{a b}  -  dE_rep/dR_k
 *   (each density-matrix column from its own atom's Krylov run; pairwise, so
 *   the forces sum to zero up to rounding).
 * F [n*3] out, FP64.
 * energies [8] out, FP64: {E_band, -TS, A = E_band - TS, E_rep,
 *   E_total = A + E_rep, N(mu), mu, 0}.
 *   E_band = 2 sum w f lam; -TS = 2 kT sum w [f ln f + (1-f) ln(1-f)];
 *   E_rep = sum over bonds i<j of phi(r_ij).
 */
tb_status tb_forces(tb_ctx* ctx, int n, const double* pos, double L,
                    const int* h_off, const int* h_idx, const double* dHblk,
                    const double* lambda, const double* S, const double* P,
                    const int* kdim, const double* mu, double* F,
                    double* energies, void* stream);

/*
 * One NVE velocity-Verlet step (fs, amu; 1 eV/(A amu) = 9.648533e-3 A/fs^2):
 *   v += dt/2 F/m;  x = wrap(x + dt v);  F = F(x) [lists .. forces];  v += dt/2 F/m.
 * pos, vel, F [n*3] in/out.  F on entry must be the force at pos.
 * energies [8] out as in tb_forces, with energies[7] = kinetic energy (eV).
 * n_electrons = 4 n.  Uses the context's own list/H/spectral buffers.
 * With group_m > 1 the Krylov stage is the m-target form (tb_group_atoms and
 * tb_krylov_density_grouped on the context's own groups, regrouped every step).
 */
tb_status tb_md_step(tb_ctx* ctx, int n, double* pos, double* vel, double* F,
                     double L, double dt_fs, double mass_amu, double* energies,
                     void* stream);

/*
 * Groups of m = group_m target atoms for the m-target form of the block
 * recursion (Sec. 3, Eq. (lanczos_blas3)); the paper leaves the grouping open,
 * this is the library's spatial reading.  The grid has g^3 cells, g the
 * largest integer with m g^3 <= n (capped at 1024); atom i lies in cell
 *   c = floor((x_i / L) * g) per component (each operation rounded, FP64),
 *   clamped to [0, g-1];
 * its key is (Morton code of c, i), the code taking bit b of c_x, c_y, c_z to
 * bits 3b, 3b+1, 3b+2.  The atoms sorted by key are cut into consecutive
 * groups of m; the last group holds the remainder.  Bit-exact.
 * pos   [n*3] FP64, each coordinate in [0, L)
 * g_off [ceil(n/m) + 1] out: group q is g_idx[g_off[q] .. g_off[q+1])
 * g_idx [n] out: the atoms in key order
 * Workspace: n ints of the context.  Any group_m in 1..4.
 */
tb_status tb_group_atoms(tb_ctx* ctx, int n, const double* pos, double L, int* g_off,
                         int* g_idx, void* stream);

/*
 * Cluster map, block Krylov space, projected eigensolve and spectral record in
 * the m-target form (Sec. 3, Eq. (lanczos_blas3)).  For each
 * group q of targets g_idx[g_off[q] .. g_off[q+1]) (1..group_m targets, any
 * partition of the atoms, e.g. from tb_group_atoms): the union of the targets'
 * clusters is formed and each target's block Krylov space is built from its own
 * four orbitals in the Hamiltonian of that union (A_k, B_k block diagonal over
 * the group, one sweep of H over all the group's columns).  The outputs, their
 * layout and the projected eigensolve are those of tb_krylov_density; with
 * groups of one target the result is tb_krylov_density's up to rounding.
 * Needs a context created with group_m >= 2 (else TB_ERR_INVALID_ARG).
 * A union larger than max_union sets TB_ERR_CAPACITY (info = its size) and
 * leaves the group's targets with an empty record; a group of a size outside
 * 1..group_m, or a target whose cluster list does not start with it, sets
 * TB_ERR_INVALID_ARG (info = the group or the target).  Atoms in no group get
 * no output.
 */
tb_status tb_krylov_density_grouped(tb_ctx* ctx, int n, int n_groups, const int* g_off,
                                    const int* g_idx, const int* c_off, const int* c_idx,
                                    const int* h_off, const int* h_idx,
                                    const double* Hblk, const float* Hsk,
                                    double* lambda, double* S, double* P, int* kdim,
                                    void* stream);

/*
 * Autotuner of the mixed path's block-Lanczos launch (the paper's cost per
 * target grows as O(n_c^3) with the cluster size n_c, Sec. 2, and clusters are
 * uneven in compressed or polymerised crystals).  On the given lists (as from
 * tb_build_neighbors / tb_assemble_H) it times, with CUDA events on `stream`:
 *   - the persistent Krylov + eigensolve queue, in index order and largest
 *     clusters first, each with two tiles (8 records per cluster slot in
 *     shared memory at 4 CTAs per SM, or 6 at 5 CTAs per SM);
 *   - separate launches per cluster-size bucket, for partitions of the
 *     observed size range into 1..TB_TUNE_MAX_BUCKETS buckets, each bucket's
 *     tile chosen among shared-memory record capacities (6 or 8 records per
 *     cluster slot) and register budgets (4 or 5 CTAs per SM) by timing that
 *     bucket alone, plus the separate eigensolver;
 * and keeps the fastest plan in the context: later calls with schedule
 * TB_SCHED_AUTO use it (the plan applies to any lists: each target goes to the
 * bucket of its cluster size).  Finally it runs the chosen plan once, so that
 * lambda, S, P, kdim hold the record of the given lists.  Synchronises the
 * stream; not capturable (tune before capturing a graph).  Mixed and BF16
 * precision with group_m == 1 only (else TB_ERR_INVALID_ARG).
 * report (host, may be NULL) receives the histogram and the choices.
 */
#define TB_TUNE_MAX_BUCKETS 4
#define TB_TUNE_BINS 128
typedef struct tb_tune_report {
  int bin_width;                               /* atoms per histogram bin (8)          */
  int n_bins;                                  /* bins in use: ceil(max_cluster / 8)   */
  int hist[TB_TUNE_BINS];                      /* targets with cluster size in
                                                * (q bin_width, (q+1) bin_width]       */
  int schedule;                                /* the chosen tb_schedule               */
  float ms_persistent;                         /* Krylov + eigensolve time, per plan   */
  float ms_persistent_largest_first;
  float ms_separate;
  float ms_bucketed;                           /* best partition into buckets          */
  int persistent_records_per_slot;             /* tile of the persistent queue in the  */
  int persistent_ctas_per_sm;                  /* context after tuning                 */
  int n_buckets;                               /* of the best bucketed plan            */
  int bucket_hi[TB_TUNE_MAX_BUCKETS];          /* bucket b: sizes (hi[b-1], hi[b]]     */
  int bucket_count[TB_TUNE_MAX_BUCKETS];       /* targets in the bucket                */
  int bucket_records_per_slot[TB_TUNE_MAX_BUCKETS];
  int bucket_ctas_per_sm[TB_TUNE_MAX_BUCKETS];
  float bucket_ms[TB_TUNE_MAX_BUCKETS];        /* the bucket's block-Lanczos launch    */
} tb_tune_report;

tb_status tb_autotune(tb_ctx* ctx, int n, const int* c_off, const int* c_idx, const int* h_off,
                      const int* h_idx, const double* Hblk, const float* Hsk, double* lambda,
                      double* S, double* P, int* kdim, tb_tune_report* report, void* stream);

/*
 * Number of kernels of this library that one force evaluation of n atoms in a
 * box of side L launches (tb_build_neighbors, [tb_group_atoms,]
 * tb_krylov_density[_grouped], tb_find_mu, tb_forces with this context's
 * configuration); memset nodes are not counted.  *count (host) out.  No GPU
 * work.  TB_ERR_NOT_RESERVED if n exceeds the reserved size.
 */
tb_status tb_ctx_kernels_per_evaluation(const tb_ctx* ctx, int n, double L, int* count);

/*
 * Stage timing (tracing aid).  When enabled, every later call records a pair of
 * CUDA events around each of its stages on its stream (as external event nodes
 * when the stream is being captured into a graph, so graph replays record them
 * too).  Stages: 0 lists, 1 assembly, 2 block Lanczos, 3 projected
 * eigensolve + spectral record, 4 mu, 5 density blocks + forces + energies,
 * 6 grouping of the targets (tb_group_atoms, m-target form only).
 * tb_profile_enable creates the events (not capturable).
 * tb_profile_read (host out ms[7]) returns the elapsed time of each stage's most
 * recent execution, or -1 for a stage not yet run; the caller synchronises first.
 */
tb_status tb_profile_enable(tb_ctx* ctx, int enable);
tb_status tb_profile_read(tb_ctx* ctx, float* ms);

/*
 * Allocation-free chemical-potential search.  The paper has no counterpart:
 * this is a deployment variant of tb_find_mu for callers that may not
 * allocate device memory (a host runtime that owns all device allocations
 * through its own pool, or code where a cudaMalloc could synchronise the
 * device at the wrong time), and therefore cannot create a tb_ctx.
 * It runs the same search as tb_find_mu with no context: its scratch (partial
 * sums of at most TB_FIND_MU_STATIC_MAX_BLOCKS blocks, one per SM, a barrier
 * counter) lives in a fixed 40 KB device array inside the library that every
 * GPU loading the library keeps until process exit.  No allocation of any kind
 * happens in the call.
 *   n, r            atoms and Krylov block order (NT = 4r, 1 <= r <= 16)
 *   lambda, S       device, as produced by tb_krylov_density
 *   kT, n_electrons, mu_tol, max_iter   as in tb_params / tb_find_mu
 *   mu_guess        device, may be NULL
 *   mu              device out: one double;  n_count: device out, may be NULL
 *   status          device out: int[2] = {tb_status code, info}, cleared on
 *                   the stream before the search; read it after the stream
 *                   has completed (timeouts, non-convergence).
 * Returns TB_ERR_INVALID_ARG for bad arguments and TB_ERR_CAPACITY when the
 * device has more SMs than TB_FIND_MU_STATIC_MAX_BLOCKS.
 * The first call on a device does a one-time set-up there (looks up the
 * array's device address, sets the kernel's shared-memory limit); make that
 * first call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents: calls whose executions overlap on the GPU
 * race with each other, so order them on one stream or synchronise.
 */
#define TB_FIND_MU_STATIC_MAX_BLOCKS 160
tb_status tb_find_mu_static(int n, int r, const double* lambda, const double* S, double kT,
                            double n_electrons, double mu_tol, int max_iter,
                            const double* mu_guess, double* mu, double* n_count, int* status,
                            void* stream);

/*
 * Virial and pressure (Sec. 5: pressure of a diamond supercell for its
 * equation of state).  Every force of tb_forces is a sum over directed bonds,
 * F_k = sum_{j in H(k)} f_kj (band term of both density-matrix columns plus
 * the pair repulsion), f_jk = -f_kj; the configurational virial is the pair form
 *   W_ab = -1/2 sum over directed bonds (k -> j) of d_a f_kj,b,   d = R_j - R_k,
 * (equal to sum_k R_k,a F_k,b for an isolated system), and the static pressure
 * P = tr W / (3 L^3).  Reads the per-bond forces that the most recent tb_forces
 * or tb_md_step left in the context, so pos, L, h_off, h_idx must be that
 * call's; after tb_md_step pass h_off = h_idx = NULL to use the context's own
 * lists (those of the step's force evaluation).  W [9] out (row-major, eV);
 * pressure [1] out (eV/A^3; 1 eV/A^3 = 160.21766 GPa), may be NULL.  Add
 * 2 KE / (3 L^3) for the kinetic part of a moving system.
 */
tb_status tb_virial(tb_ctx* ctx, int n, const double* pos, double L, const int* h_off,
                    const int* h_idx, double* W, double* pressure, void* stream);

/*
 * Weak-coupling (Berendsen) NPT for the C60 polymerisation runs of Sec. 4
 * (MD at 25 GPa and 500 K; the paper names neither thermostat nor barostat).
 * Call after tb_md_step (box L) and tb_virial on that step's bonds, on the same
 * stream; with the step's kinetic energy KE = energies[7] and virial W:
 *   T = 2 KE / (k_B (3n - 3)),  P = (tr W + 2 KE) / (3 L^3),
 *   lambda = sqrt(1 + (dt/tau_T) (T0/T - 1))   (lambda = 1 when T = 0),
 *   mu = [1 - beta (dt/tau_P) (P0 - P)]^(1/3),
 *   v <- lambda v;  x <- mu x (kept in [0, mu L));  L <- mu L.
 * so the rescaled temperature is T + (dt/tau_T)(T0 - T) and the volume changes
 * by -beta (dt/tau_P)(P0 - P) relative.  The next tb_md_step takes the box
 * *L_new (copy it to the host) and the forces F of the unscaled configuration
 * for its first half kick (the usual weak-coupling approximation; |mu - 1| is
 * ~1e-5 per step).
 * pos, vel [n*3] in/out (device, FP64); W [9], energies [8] in (device);
 * L_new [1] out (device); state [4] out (device): T (K), P (eV/A^3), lambda, mu.
 * T0 >= 0 (K); P0 (eV/A^3; 1 GPa = 1/160.21766 eV/A^3); dt_fs < tau_T_fs,
 * dt_fs < tau_P_fs (fs); beta > 0 (A^3/eV, the barostat's compressibility).
 * Returns TB_ERR_INVALID_ARG for arguments outside these ranges.  On the
 * device, a factor that is not a positive finite number leaves pos, vel and
 * the box unchanged and sets the status word: TB_ERR_NONFINITE when a factor
 * is NaN or infinite (non-finite kinetic energy or virial), TB_ERR_INVALID_ARG
 * when it is finite but not positive (the target state too far from the
 * current one for the coupling constants), info 0 for lambda^2, 1 for mu^3.
 * Capturable.
 */
tb_status tb_npt_berendsen(tb_ctx* ctx, int n, double* pos, double* vel, double L,
                           const double* W, const double* energies, double T0, double P0,
                           double dt_fs, double tau_T_fs, double tau_P_fs, double beta,
                           double* L_new, double* state, void* stream);

/*
 * Exact gradient of the truncated local free energy (differentiable form
 * of the method).  Sec. 3: once the Krylov order reaches the minimal-polynomial
 * degree (r = r_min) the block Krylov space of a target is invariant and its
 * projection is exact, so the target's spectral record is that of the dense
 * eigen-decomposition of its cluster Hamiltonian H_c = Z diag(lam) Z^T
 * (Sec. 2).  These calls evaluate that limit directly:
 *   A_loc = sum_i A_i,  A_i = Omega_i + mu N_i,
 *   Omega_i = 2 sum_a <i a| omega(H_c(i)) |i a>,  omega(e) = -kT ln(1 + e^{-(e-mu)/kT}),
 * with mu fixed by sum_i N_i = N_e, and its exact gradient at fixed N_e
 *   dOmega_i/dH_c = 2 Z (Gamma o S^T S) Z^T,   S = Z[0:4, :],
 *   Gamma_mk = (omega(lam_m) - omega(lam_k)) / (lam_m - lam_k),  Gamma_mm = f(lam_m)
 * (Daleckii-Krein), contracted with dH/dR over the bonds of every cluster.
 * Clusters must hold at most TB_LOCAL_MAX_DIM / 4 atoms (max_cluster of the
 * context <= 128).  Precision: TB_PREC_FP64 runs everything in FP64;
 * TB_PREC_MIXED runs the dense eigen-decomposition and the W = Z M product in
 * FP32, with eigenvalues (FP64 Rayleigh quotients on the tridiagonal form),
 * divided differences, mu, energies and force sums in FP64.
 *
 * tb_ctx_reserve_local: allocates the dense workspace (one slot per SM: three
 * matrices of 4*max_cluster squared plus scratch; ~7 x 2 MB per SM in FP64 at
 * max_cluster 128) and per-target force terms for n atoms.  Not capturable.
 * Returns TB_ERR_CAPACITY if max_cluster > 128.
 *
 * With ND = 4 * max_cluster:
 * tb_local_forward: lists and bond blocks as produced by tb_build_neighbors and tb_assemble_H (Hblk FP64);
 *   lambda [n*ND] out, S [n*4*ND] out (layout of tb_krylov_density with NT = ND;
 *   entries beyond 4 n_c(i) are 0), kdim [n] out (= 4 n_c(i));
 *   Zstore (may be NULL): [n*ND*ND] elements of the context precision (double
 *   for TB_PREC_FP64, float for TB_PREC_MIXED), out: target i's eigenvectors
 *   at i*ND*ND, row-major with leading dimension 4 n_c(i) (the stored-basis
 *   backward); mu (device, out): one double; energies [8] out as in tb_forces
 *   (A = A_loc, E_total = A_loc + E_rep).
 * tb_local_gradient: F [n*3] out = -d(A_loc + E_rep)/dR at the given mu (the
 *   forward's), from the forward's lambda and S; if Zstore is NULL the
 *   eigenvectors are recomputed (same arithmetic, same bits), else read.
 * Cluster capacity overflow and non-finite values go to the status word.
 */
#define TB_LOCAL_MAX_DIM 512
tb_status tb_ctx_reserve_local(tb_ctx* ctx, int n_atoms);
tb_status tb_local_forward(tb_ctx* ctx, int n, const double* pos, double L, const int* c_off,
                           const int* c_idx, const int* h_off, const int* h_idx,
                           const double* Hblk, double* lambda, double* S, int* kdim,
                           void* Zstore, double* mu, double* energies, void* stream);
tb_status tb_local_gradient(tb_ctx* ctx, int n, const double* pos, double L, const int* c_off,
                            const int* c_idx, const int* h_off, const int* h_idx,
                            const double* Hblk, const double* dHblk, const double* lambda,
                            const double* S, const void* Zstore, const double* mu, double* F,
                            void* stream);

/* Library version string (static, host). */
const char* tb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TB_H */
