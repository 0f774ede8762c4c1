/*
 * gint — real-space grid integration for LCAO (numerical atomic orbital) Kohn-Sham DFT on
 * one NVIDIA GB300 (sm_103a).  C ABI: plain pointers and sizes, no C++ or framework types.
 *
 * What is computed (paper: "ABACUS: An Electronic Structure Analysis Package for the AI
 * Era", Sec. IV.A-D):
 *   basis     phi_mu(r) = f_{zeta l}(|r - tau_I|) Y_lm(r_hat): a strictly localised radial
 *             function times a real spherical harmonic (Sec. IV.A; the same "radial times
 *             spherical harmonic" form the paper states for projectors and auxiliary functions).
 *   vlocal    V_mu,nu(R) = Sum_r phi_mu(r - tau_I) V(r) phi_nu(r - tau_J - R) dV — the
 *             two-centre template O_mu,nu(R) of Sec. IV.B with a multiplicative local
 *             operator, evaluated on the uniform real-space grid ("grid integration", Sec. IV.B),
 *             stored in a sparse block container (the paper's HContainer, Fig. 2 caption).
 *   rho       rho(r) = Sum_R Sum_mu,nu rho_mu,nu(R) phi_mu(r) phi_nu(r - R), the real-space
 *             density from the density matrix of Eq. (density_matrix), Sec. IV.B; it is the
 *             adjoint of vlocal: <rho(r), V(r)> dV = Sum rho_mu,nu V_mu,nu (Eq. lcao_etot2).
 *   force     the basis-motion (Pulay) term of Eq. (force_lcao), Sec. IV.D, for
 *             L = Sum_blocks Sum_mu,nu rho_mu,nu(R) V_mu,nu(R) with V(r) held fixed:
 *             F_I = -dL/dtau_I.
 *
 * Conventions.
 *   cell      rows a1, a2, a3 (bohr), row-major double[9].
 *   grid      N1 x N2 x N3; point (i,j,k) sits at r = (i/N1) a1 + (j/N2) a2 + (k/N3) a3; grid
 *             arrays (V, rho) are double, C order (i, j, k) with k fastest; dV = |det A|/(N1 N2 N3).
 *   atoms     tau is Cartesian (bohr) and used as given (it need not lie inside the cell).
 *   orbitals  per species: radial functions in the order given, each with 2l+1 real harmonics
 *             ordered m = 0, +1, -1, +2, -2 (no Condon-Shortley phase; l = 1 is
 *             sqrt(3/4pi) (z, x, y)/r); l <= 2.  Radials are clamped cubic splines through the
 *             table f(i*dr), end slopes f'(0) (given) and 0 at the last knot, and f = 0 for
 *             r >= rcut.  At r = 0 the orbital takes its limit (f(0) Y_00 for l = 0, else 0).
 *   blocks    a block key (I, J, n1, n2, n3) couples phi centred at tau_I with phi centred at
 *             tau_J + n1 a1 + n2 a2 + n3 a3; it exists iff that distance is below
 *             rcut_I + rcut_J.  Keys are sorted by (I, J, n1, n2, n3); block b holds
 *             norb_I x norb_J doubles, row-major, at offsets[b].  H and the density matrix
 *             use this layout.  The partner of (I,J,R) is (J,I,-R); V_mu,nu(R) = V_nu,mu(-R).
 *
 * Execution and errors.  Every compute call is asynchronous on the given CUDA stream
 * (a cudaStream_t passed as void*; NULL = legacy default stream) and reads/writes only
 * caller-owned device buffers plus library-owned memory created in gint_setup.  Inputs are
 * validated on the host before any launch; a failed validation returns GINT_EINVAL and
 * launches nothing.  Kernels bound every wait; a wait that runs out records GINT_ETIMEOUT in
 * a device status word that gint_get_status() reads.  There is no CPU fallback: without a usable
 * sm_103a device gint_setup returns GINT_ECUDA.  gint_last_error() gives a message for the
 * last failing call on the calling thread.
 */
#ifndef GINT_H
#define GINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gint_handle_s *gint_handle;

typedef enum {
    GINT_OK = 0,
    GINT_EINVAL = 1,    /* bad argument: null pointer, size, shape, l > 2, limits */
    GINT_ENOMEM = 2,    /* device or host allocation failed */
    GINT_ECUDA = 3,     /* CUDA runtime error or no sm_103a device */
    GINT_ETIMEOUT = 4,  /* a kernel gave up on a bounded wait (device status word) */
    GINT_ESTATE = 5     /* call not valid for this handle's state (e.g. topology changed) */
} gint_status;

/* Arithmetic of the per-batch contraction.  Orbital values, the contraction and the
 * per-batch partial sums use the named precision; the accumulation across batches into the
 * block store, rho(r) and the forces is FP64 in every mode.
 *   GINT_FP64    FP64 CUDA-core FMA throughout (orbitals evaluated in FP64).
 *   GINT_FP32    FP32 CUDA-core FMA (orbitals in FP32).
 *   GINT_TF32X3  tcgen05 tensor cores, kind::tf32, each FP32 operand split hi+lo and
 *                hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory.
 *   GINT_BF16X3  tcgen05 kind::f16 with bf16 hi+lo splits, 3 products (about 16 bits).
 *   GINT_BF16X6  tcgen05 kind::f16 with bf16 hi+mid+lo splits, the 6 products of order <= 2.
 *   GINT_FP16X3  tcgen05 kind::f16 with fp16 hi+lo splits, 3 products: the 11-bit significand of
 *                TF32 per term (about 22 bits in all, as GINT_TF32X3) at the f16 tensor rate.
 *                fp16's narrow exponent is handled by exact power-of-two scaling: orbital values
 *                by a bound from the radial tables, V(r) dV and the density matrix by their
 *                largest magnitude in the call, so the largest term sits near 2^14; values more
 *                than 2^17 below that largest one keep an absolute accuracy of about 2^-39 of
 *                it instead of a relative one. */
typedef enum {
    GINT_FP64 = 0,
    GINT_FP32 = 1,
    GINT_TF32X3 = 2,
    GINT_BF16X3 = 3,
    GINT_BF16X6 = 4,
    GINT_FP16X3 = 5
} gint_prec;

/* One atomic species.  All pointers are host memory, read during gint_setup only. */
typedef struct {
    int nrad;              /* number of radial functions, 1..16 */
    const int *l;          /* [nrad] angular momentum of each radial, 0..2 */
    double rcut;           /* cutoff radius (bohr), > 0 */
    double dr;             /* table spacing (bohr), > 0 */
    int ntab;              /* knots per radial; (ntab-1)*dr must reach rcut */
    const double *ftab;    /* [nrad * ntab] f(i*dr), radial-major */
    const double *dfdr0;   /* [nrad] slope f'(0) of each radial */
} gint_species;

typedef struct {
    int batch[3];          /* grid points per vlocal batch along a1, a2, a3 (default 4, 4, 4);
                              at most 16 per axis and 128 in all, even along a3 */
    int batch_rho[3];      /* grid points per rho/force batch (default 4, 4, 8), same limits.
                              Batches whose orbital count (256) or atom-image count (64)
                              exceeds the kernel limits are split. */
    int wait_budget;       /* clock cycles a tensor-core kernel waits on one pipeline barrier
                              before it gives up with GINT_ETIMEOUT; 0 = default (4e9, about
                              2 s).  The final wait for in-flight MMAs always uses the default. */
    int reserved;
} gint_options;

/* Sizes of a handle (host values). */
typedef struct {
    int64_t npts;          /* N1*N2*N3 */
    int64_t nblocks;       /* blocks in the store */
    int64_t nvalues;       /* doubles in the store */
    int64_t nbatches;      /* vlocal grid batches */
    int64_t nslots;        /* vlocal (batch, atom image) pairs */
    int max_orbitals;      /* largest vlocal per-batch orbital count */
    int max_slots;         /* largest vlocal per-batch atom-image count */
    double dV;             /* volume element */
    double flops_useful;   /* 2 * Sum_r n(r)^2: one contraction, n(r) = orbitals whose sphere holds r */
    double flops_dense;    /* 2 * Sum_b npts_b * nb_b^2: the dense vlocal per-batch contraction */
    int64_t nbatches_rho;  /* rho/force grid batches */
    int max_orbitals_rho;  /* largest rho/force per-batch orbital count */
    int nbasis;            /* orbitals of the cell, Sum_I norb(I) (dense k-space matrix order) */
    double flops_dense_rho;/* 2 * Sum_b npts_b * nb_b^2 over the rho/force batches */
} gint_info_t;

/* Build a handle: validates the inputs, fits the radial splines, finds the block list
 * (Sec. IV.B: pairs (I, J, R) over all valid neighbouring cells) and the batch -> atom-image
 * lists (strict locality of NAOs, Sec. IV.A), and uploads them to the current device.
 * natoms >= 1, nspecies >= 1, species[i] in [0, nspecies), grid[i] >= 1; opt may be NULL.
 * All pointers are host memory.  On success *out owns device memory until gint_destroy. */
gint_status gint_setup(gint_handle *out, const double cell[9], int natoms, const int *species,
                       const double *tau, int nspecies, const gint_species *sp,
                       const int grid[3], const gint_options *opt);

/* Release everything the handle owns.  NULL is accepted. */
gint_status gint_destroy(gint_handle h);

/* Read-only host view of the block layout: keys[5*b .. 5*b+4] = (I, J, n1, n2, n3),
 * offsets[b] (nblocks+1 entries, offsets[nblocks] = nvalues).  Valid until gint_destroy or
 * gint_update_positions. */
gint_status gint_block_layout(gint_handle h, int64_t *nblocks, int64_t *nvalues,
                              const int32_t **keys, const int64_t **offsets);

/* The handle's description.  After gint_update_positions, the first call counts flops_useful
 * again for the new positions (a host pass over every grid point of the vlocal batches). */
gint_status gint_get_info(gint_handle h, gint_info_t *info);

/* Move the atoms (host tau, natoms*3).  The block list (and with it the layout of H and of the
 * density matrix) must stay the same: if some pair enters or leaves the cutoff, nothing changes
 * and GINT_ESTATE is returned (build a new handle).  The batch -> atom-image lists are rebuilt
 * for the new positions on the host (in parallel over host threads); a batch that keeps its
 * list keeps its slot-pair tables, one whose list changed takes the entries of the atom images
 * it kept from its old table and looks the others up.  A decomposition whose lists are all
 * unchanged keeps its device arrays and tables and receives the new slot positions only, one
 * whose lists changed is copied into its device arrays again (an array too small for the new
 * lists is replaced by a larger one).  The result equals a handle set up at the new positions.
 * The handle keeps the host arrays an update replaced, as storage for the next one (host memory
 * about twice the lists').  Blocking: the call synchronises with the device before
 * replacing arrays.  A multi-structure job (gint_batch_create) copies the lists when it is
 * created: create it again after a move. */
gint_status gint_update_positions(gint_handle h, const double *tau);

/* H <- V_mu,nu(R) for the potential V (device, npts doubles).  H (device, nvalues doubles)
 * is overwritten; both halves of every partner pair are written. */
gint_status gint_vlocal(gint_handle h, const double *V_dev, double *H_dev, gint_prec prec,
                        void *stream);

/* rho (device, npts doubles) <- rho(r) from the density matrix DM (device, block layout).
 * Only the block-symmetric part of DM contributes. */
gint_status gint_rho(gint_handle h, const double *DM_dev, double *rho_dev, gint_prec prec,
                     void *stream);

/* F (device, natoms*3 doubles) <- F_I = -dL/dtau_I, L = Sum DM_mu,nu V_mu,nu(R), for V
 * (device, npts) and DM (device, block layout).  DM is symmetrised in the block sense first
 * (into library-owned scratch), so any DM is accepted. */
gint_status gint_force(gint_handle h, const double *V_dev, const double *DM_dev, double *F_dev,
                       gint_prec prec, void *stream);

/* rho and F from one pass over the grid (the backward of vlocal); either output may be NULL. */
gint_status gint_rho_force(gint_handle h, const double *V_dev, const double *DM_dev,
                           double *rho_dev, double *F_dev, gint_prec prec, void *stream);

/* Strain derivative of L = Sum_blocks Sum_mu,nu DM_mu,nu V_mu,nu(R), the grid part of the
 * stress of Eq. stress (sigma_ab = -(1/Omega) dE/deps_ab, Sec. III; the LCAO stress follows
 * the force formulas, Sec. IV.D).  A homogeneous strain maps every vector x -> (1 + eps) x:
 * cell, atoms, lattice translations and grid points (fractional grid coordinates fixed); the
 * grid values of V are held fixed and dV scales with det(1 + eps).  Then
 *   dL/deps_ab = delta_ab dV Sum_r V rho(r)
 *              + 2 dV Sum_r V(r) Sum_mu d/dx_a phi_mu(d_mu) (d_mu)_b (Phi sym(DM))_r,mu
 * with d_mu = r - tau_I - R the displacement from the orbital's centre.
 *   V      device, npts doubles;   DM  device, block layout (symmetrised in the block sense)
 *   dLde   device, 9 doubles, row-major [a][b], overwritten
 * Asynchronous on `stream`; errors as gint_force. */
gint_status gint_strain_derivative(gint_handle h, const double *V_dev, const double *DM_dev,
                                   double *dLde_dev, gint_prec prec, void *stream);

/* Folding into momentum space (Sec. IV.B): Xk[q] = Sum_R X(R) exp(i k_q.R) for the block store
 * X (device, block layout), R = n1 a1 + n2 a2 + n3 a3 of each block key, k_q.R = 2 pi kappa_q.n.
 *   kfrac  host, nk x 3: k points in fractional reciprocal coordinates kappa; 1 <= nk <= 4096
 *   Xk     device, nk x nbasis x nbasis complex numbers (re, im interleaved, row-major, rows
 *          = orbital mu in atom-major order, see gint_info_t.nbasis), overwritten; entries of
 *          atom pairs without a block are zero
 * Asynchronous on `stream` (the k points are copied before the call returns). */
gint_status gint_fold(gint_handle h, const double *X_dev, int nk, const double *kfrac, double *Xk_dev,
                      void *stream);

/* The inverse direction (Eq. density_matrix with Xk = Sum_n f c c*): X(R) = Re Sum_q w_q Xk[q]
 * exp(-i k_q.R) for every block of the store; with w_q = 1/N_k on a complete k mesh it inverts
 * gint_fold.  Xk as in gint_fold (device, read); kfrac, w host (nk x 3, nk); X (device, block
 * layout) overwritten. */
gint_status gint_unfold(gint_handle h, const double *Xk_dev, int nk, const double *kfrac, const double *w,
                        double *X_dev, void *stream);

/* Density matrix from Kohn-Sham eigenvectors, Eq. density_matrix:
 *   DM_mu,nu(R) = Re Sum_q w_q Sum_n f_n,q c_n,mu,q c*_n,nu,q exp(-i k_q.R)
 * for every block (I, J, R) of the store (k_q.R = 2 pi kappa_q.n; w_q = 1/N_k in the paper).
 *   kfrac, w  host, nk x 3 and nk
 *   C         device, nk x nbasis x nbands complex numbers (re, im interleaved), row-major:
 *             row = orbital mu (atom-major order), column = band n
 *   f         device, nk x nbands occupations
 *   DM        device, block layout, overwritten
 * prec: GINT_FP64 (CUDA-core complex GEMM per k point) or GINT_TF32X3 (tensor cores: the band
 * sum in 64-term segments accumulated in TMEM, segments added in FP32; relative error ~6e-7).
 * Library-owned scratch of 16 * nbasis^2 bytes (dense rho(k)) is allocated on first use and kept
 * until gint_destroy. */
gint_status gint_density_matrix(gint_handle h, int nk, const double *kfrac, const double *w, int nbands,
                                const double *C_dev, const double *f_dev, double *DM_dev, gint_prec prec,
                                void *stream);

/* Backward of gint_vlocal for L = Sum_blocks Sum_mu,nu gH_mu,nu V_mu,nu(R) (gH: device, block
 * layout, e.g. the incoming gradient of H):
 *   gV (device, npts)       <- dL/dV(r)   = dV * rho(r) built from the block-symmetric part of gH
 *   gtau (device, natoms*3) <- dL/dtau_I  = -F_I (the Pulay term of Eq. force_lcao with V fixed)
 * i.e. the adjoint of vlocal (Eq. lcao_etot2) and its basis-motion derivative (Sec. IV.D).
 * Either output may be NULL. */
gint_status gint_vlocal_backward(gint_handle h, const double *V_dev, const double *gH_dev,
                                 double *gV_dev, double *gtau_dev, gint_prec prec, void *stream);

/* out[0] (device double) <- Sum_r rho(r) dV, summed in FP64 on the device. */
gint_status gint_charge(gint_handle h, const double *rho_dev, double *out_dev, void *stream);

/* out[0] (device double) <- Sum_i A[i] B[i] over the block store (e.g. Tr(rho S),
 * <rho_mu,nu, V_mu,nu>), FP64 on the device. */
gint_status gint_block_dot(gint_handle h, const double *A_dev, const double *B_dev,
                           double *out_dev, void *stream);

/* out[0] (device double) <- Sum_i A[i] B[i] over the block store, like gint_block_dot, but
 * without allocating anything: for callers that cannot allocate device memory at the call
 * site (inside an allocator or memory-pool callback, or after a fixed memory budget has been
 * reached).  The paper has no counterpart; this is a service of the library.  Partial sums
 * live in a static device array of 1024 doubles that every GPU loading the library holds
 * until exit; a store of more than 1024 * 65536 values is rejected with GINT_EINVAL.  Each
 * call looks up the array's address in the current context.  Errors: GINT_EINVAL for a null
 * argument or a device other than the handle's.  All calls share the array: calls that
 * overlap on the GPU race.  A, B, out: device memory. */
gint_status gint_block_dot_noalloc(gint_handle h, const double *A_dev, const double *B_dev,
                                   double *out_dev, void *stream);

/* End-to-end call from host buffers: copies V and DM (pinned or pageable host memory) to
 * library-owned device buffers, runs vlocal and rho_force on `stream`, and copies H, rho and F
 * back.  DM comes in while vlocal runs and H goes out while rho_force runs, on a copy stream
 * the library creates on the first call (overlap needs pinned host memory).  Synchronous:
 * returns after the results are in host memory.  Outputs may be NULL. */
gint_status gint_run_host(gint_handle h, const double *V_host, const double *DM_host,
                          double *H_host, double *rho_host, double *F_host, gint_prec prec,
                          void *stream);

/* A reusable multi-structure job (Sec. IV.B grid integrals of many independent structures):
 * every structure's grid batches are concatenated into one work list, run by one persistent
 * launch of the tensor-core vlocal kernel (two when some structures have batches of more than
 * 192 orbitals, which need the single-accumulator layout) and one of the rho kernel; the sequence
 * (H zeroing, density-matrix conversion, the two persistent launches, block mirroring) is
 * captured once into a CUDA graph that gint_batch_launch replays.  prec must be a tensor-core
 * precision (GINT_TF32X3, GINT_BF16X3, GINT_BF16X6, GINT_FP16X3); at most 255 structures, all on the current
 * device, at most 8 distinct species in total.  Pointer arrays are host memory, read during
 * create; the buffers they point to are device memory and are bound to the job.  DM and rho
 * may be NULL (vlocal only).  The handles must outlive the job.  A handle may appear more than
 * once: spin channels are entries that share one geometry (collinear spin: V_up / V_down with
 * DM_up / DM_down; non-collinear: the four real components V_uu, V_dd, Re V_ud, Im V_ud with the
 * matching density-matrix components: the spin densities of Sec. II.A (exchange-correlation
 * functionals) and the 2x2 spinor potential of its non-collinear subsection); every repeated
 * occurrence gets a private FP32 density-matrix buffer owned by the job. */
typedef struct gint_batch_s *gint_batch;
gint_status gint_batch_create(gint_batch *out, int nstruct, const gint_handle *hs,
                              const double *const *V, double *const *H, const double *const *DM,
                              double *const *rho, gint_prec prec);
/* Replay the job's graph on `stream` (asynchronous). */
gint_status gint_batch_launch(gint_batch b, void *stream);
gint_status gint_batch_destroy(gint_batch b);

/* Choose batch shapes for one structure by timing candidates on the current device: vlocal
 * shapes of at most 64 points (the tensor-core accumulation error grows with the MMA steps per
 * batch; for GINT_FP16X3, whose steps are 16 points deep, up to 128) and rho shapes of 128
 * points (one M = 128 tile).  Inputs as for gint_setup; writes
 * the fastest shapes into *best (and their times in ms, if the pointers are non-NULL).
 * Allocates and frees its own device buffers. */
gint_status gint_autotune(const double cell[9], int natoms, const int *species, const double *tau,
                          int nspecies, const gint_species *sp, const int grid[3], gint_prec prec,
                          gint_options *best, double *ms_vlocal, double *ms_rho);

/* One-shot form of the multi-structure job: for each s, H[s] <- vlocal(V[s]) and, if DM and
 * rho are non-NULL, rho[s] <- rho(DM[s]).  With a tensor-core precision this is
 * gint_batch_create + gint_batch_launch + a stream synchronisation + gint_batch_destroy (so it
 * blocks); with GINT_FP64 / GINT_FP32 the structures run one after another on the CUDA cores. */
gint_status gint_batched(int nstruct, const gint_handle *hs, const double *const *V,
                         double *const *H, const double *const *DM, double *const *rho,
                         gint_prec prec, void *stream);

/* Status word of the handle's kernels (GINT_OK or GINT_ETIMEOUT); synchronises the stream
 * the handle last used.  Clears the word. */
gint_status gint_get_status(gint_handle h);

/* Message for the last failing call on this thread ("" if none). */
const char *gint_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
