/*
 * fla.h -- C interface of the GB300 (sm_103a) library for the fully Lagrangian
 * approach (FLA) advance and the interphase source-term deposits of
 * Stafford & Rybdylova, "Interphase coupling for gas-droplet flows using the
 * fully Lagrangian approach".  Equation numbers below are the paper's.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Domain [0,1]^dim (dim = 2 or 3) with a uniform mesh of n^dim cells, cell
 *    size dx = 1/n, cell centres (i + 1/2) dx.  Cells and mesh nodes are
 *    numbered with x fastest, then y, then z.
 *  - Every pointer named *_dev is device memory that the CALLER owns and keeps
 *    alive until the work enqueued on the stream has finished.  The library
 *    never allocates device memory in these calls; temporary storage comes from
 *    the caller's workspace (see fla_workspace_size).  Only fla_create
 *    allocates (a small status block) and fla_destroy frees it.
 *  - All GPU work is enqueued asynchronously on the caller's stream; a NULL
 *    stream is the legacy default stream.  A return of FLA_OK means that the
 *    arguments were valid and the kernels were enqueued.  Problems found on
 *    the device (non-finite values) are counted in a status block that only
 *    fla_sync_status reads back.  Device code never traps or asserts.
 *  - Host-detectable errors return a negative fla_status and enqueue nothing.
 *  - There is no CPU fallback: without a usable CUDA device fla_create returns
 *    FLA_ERR_CUDA.
 */
#ifndef FLA_H
#define FLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLA_ABI_VERSION 11

/* cudaStream_t without including the CUDA headers. */
typedef struct CUstream_st* fla_stream_t;

typedef enum {
    FLA_OK = 0,
    FLA_ERR_ARG = -1,          /* invalid argument: null pointer, bad size or mode */
    FLA_ERR_CUDA = -2,         /* a CUDA runtime call or kernel launch failed */
    FLA_ERR_WORKSPACE = -3,    /* workspace pointer missing, misaligned or too small */
    FLA_ERR_NONFINITE = -4,    /* reported by fla_sync_status: non-finite records seen */
    FLA_ERR_TIMEOUT = -5,      /* a bounded device-side wait ran out (fla_sync_status) */
    FLA_ERR_UNSUPPORTED = -6   /* valid but not implemented combination */
} fla_status;

/* Arithmetic and storage type of a cloud.  FLA_F32X2 ("compensated" single
 * precision) stores every state value as an unevaluated sum hi + lo of two
 * floats (about 48 significant bits): state_dev holds the n_planes hi planes
 * of the FLA_F32 layout followed by n_planes lo planes, and fla_advance
 * integrates in double-float arithmetic on the single-precision pipe from
 * double-float carrier nodes (fla_carrier_sample with FLA_F32X2).  Cell keys,
 * records, deposits and their outputs are single precision (from the hi
 * planes), except det J and n = n0/|det J|, which the records form in double
 * precision from hi + lo.  Near a fold caustic n is ill-conditioned: single
 * precision anywhere in the trajectory (seed position, interpolated carrier,
 * stage arithmetic) moves det J there by far more than its size, and this form
 * keeps the sources within 1e-4 of the double-precision method. */
enum { FLA_F32 = 0, FLA_F64 = 1, FLA_F32X2 = 2 };
enum { FLA_CLOUD_FLA = 0, FLA_CLOUD_LPT = 1 };        /* FLA seeds (with J) or plain parcels */
enum { FLA_KERNEL_ISO = 0, FLA_KERNEL_ANISO = 1 };    /* deposit kernel shape */

/* Analytic carriers sampled onto the mesh nodes (stand-ins for the paper's
 * Navier-Stokes carrier of Eq. 1). */
enum {
    FLA_CARRIER_UNIFORM = 0,   /* u = U */
    FLA_CARRIER_LINEAR = 1,    /* u = U + A (x - xref) */
    FLA_CARRIER_TG2 = 2,       /* (sin pi x cos pi y, -cos pi x sin pi y) */
    FLA_CARRIER_JETVORT2 = 3,  /* planar jet exp(-((y-1/2)/w)^2) e_x + Lamb-Oseen vortices */
    FLA_CARRIER_ABCJET3 = 4    /* ABC flow at wavenumber 2 pi + round jet along z */
};

/* Per-droplet meta word: release index in bits 0..23 plus state bits.
 * A seed with neither ACTIVE nor DEAD set is pending (not yet released).
 * FOLD marks a droplet of a single-precision FLA cloud whose J and W are
 * currently integrated in double precision (see fla_cloud.fold_dev). */
#define FLA_META_BATCH_MASK 0x00FFFFFFu
#define FLA_META_FOLD 0x20000000u
#define FLA_META_DEAD 0x40000000u
#define FLA_META_ACTIVE 0x80000000u

#define FLA_MAX_VORTICES 16
#define FLA_NO_DEADLINE 2147483647

/* Opaque context: the device it was created on, its SM count and a small
 * device status block. */
typedef struct fla_ctx fla_ctx;

typedef struct {
    int32_t dim;               /* 2 or 3 */
    int32_t n;                 /* cells per axis, >= 1; n^dim < 2^31 */
} fla_mesh;

typedef struct {
    int32_t kind, dim;
    double U[3];
    double A[9];               /* row-major: u_i += A[3 i + j] (x_j - xref_j) */
    double xref[3];
    int32_t n_vortex;          /* <= FLA_MAX_VORTICES */
    double vortex[FLA_MAX_VORTICES][5]; /* x0, yc, Gamma, rc, Uadv: centre x = frac(x0 + Uadv t) */
    double jet_width;          /* planar jet width w */
    double abc[3];             /* ABC amplitudes A, B, C */
    double jet_amp, jet_radius;/* round jet u_z += amp exp(-(rho/radius)^2) */
} fla_carrier_desc;

/* One release ("batch") of seeds.  32 bytes, device array. */
typedef struct {
    double St0;                /* Stokes number at release (Eq. 5 with r = r0) */
    double n0;                 /* FLA: number density at release (Eq. 6, App. A);
                                  LPT: real droplets represented by one parcel */
    double h0;                 /* FLA: smoothing length at release (Eq. 15) */
    int32_t step_start;        /* step index at which the seeds are released */
    int32_t step_dead;         /* step index from which they are inactive (evaporated) */
} fla_batch;

/* A cloud of droplets stored as structure-of-arrays "planes" of 4 values:
 * state_dev holds n_planes * n * 4 values of the cloud's dtype; value c of
 * droplet i in plane p is at index (p * n + i) * 4 + c.  The flattened value
 * vector of one droplet is
 *   FLA: x[dim], v[dim], J[dim*dim], W[dim*dim], acc[1+dim], zero padding
 *   LPT: x[dim], v[dim], acc[1+dim], zero padding
 * (J = dx/dx0 row-major, W = dJ/dt, acc = window sums of mdot and F + mdot v).
 * Use fla_state_layout for n_planes and the offsets.  Pending seeds hold
 * their release position in x. */
typedef struct {
    int32_t kind;              /* FLA_CLOUD_FLA or FLA_CLOUD_LPT */
    int32_t dim;
    int32_t dtype;             /* FLA_F32, FLA_F64 or FLA_F32X2 */
    int32_t n_batches;
    int64_t n;                 /* droplets, < 2^31 */
    void* state_dev;
    uint32_t* meta_dev;        /* n meta words */
    const fla_batch* batches_dev; /* n_batches entries */
    double delta;              /* d^2-law rate: r^2 = r0^2 + delta (t - t0), r0 = 1 (Eq. 4) */
    /* Fold guard of single-precision FLA clouds (NULL: none).  Near a fold
     * caustic det J passes through zero (Eq. 6 gives n -> infinity) and its
     * single-precision value loses its relative accuracy.  With fold_dev set,
     * fla_advance moves a droplet whose |det J| drops below tau_fold to double
     * precision for the J and W part of its RK4 step, keeping those values in
     * fold_dev (FP64 planes of 4: J[dim*dim] then W[dim*dim]; value c of
     * droplet i in plane p at (p * n + i) * 4 + c; fla_fold_bytes gives the
     * size) and setting FLA_META_FOLD; it moves back once |det J| exceeds
     * 4 tau_fold.  The single-precision J and W in state_dev stay the rounded
     * copies.  Records of flagged droplets take det J and 1/|det J| from
     * fold_dev in double precision.  Caller-owned, 16-byte aligned; the
     * library reads it only for flagged droplets, so it needs no clearing. */
    void* fold_dev;
    double tau_fold;           /* fold threshold on |det J| (> 0 when fold_dev is set); 1e-2 typical */
} fla_cloud;

/* Bytes of fold_dev for n droplets of dimension dim. */
size_t fla_fold_bytes(int32_t dim, int64_t n);

/* Kernel-regression deposit settings. */
typedef struct {
    int32_t kernel;            /* FLA_KERNEL_ISO: Eq. 14 with h of Eq. 15;
                                  FLA_KERNEL_ANISO: covariance f h0^2 J J^T + h_min^2 I */
    int32_t per_cell;          /* 0: sources per unit volume; 1: multiplied by the cell volume */
    double h_min, h_max;       /* smoothing-length clamps (absolute lengths), 0 < h_min <= h_max */
    double p;                  /* h = h0 |det J|^p; the paper's Eq. 15 is p = 1 */
    double window_dt;          /* time covered by the window sums acc (> 0) */
    int32_t precision;         /* single-precision clouds: FLA_PREC_MIXED (det J and 1/|det J| in
                                  double where they can cancel, and from fold_dev for flagged droplets)
                                  or FLA_PREC_PLAIN (det J, 1/|det J| in single precision throughout);
                                  ignored by double-precision clouds */
    int32_t reserved;          /* 0 */
    const void* mlp_dev;       /* packed learned correction (fla_mlp_pack), or NULL for the plain
                                  method; single-precision clouds with FLA_KERNEL_ISO only */
    float* mlp_out_dev;        /* optional (with mlp_dev): g(f_i) per droplet index (n floats);
                                  entries of droplets that are not deposited are left as they are */
} fla_deposit_cfg;

enum { FLA_PREC_MIXED = 0, FLA_PREC_PLAIN = 1 };

/* Deposit outputs, device arrays of the cloud's dtype, n_cells entries each
 * (s_mom: dim consecutive planes of n_cells).  dsum_dev (the kernel-estimator
 * denominator) may be NULL. */
typedef struct {
    void* s_mass_dev;
    void* s_mom_dev;
    void* dsum_dev;
} fla_sources;

typedef struct {
    uint32_t* counts_dev;      /* parcels per cell, n_cells entries */
    void* s_mass_dev;          /* n_cells of the cloud dtype */
    void* s_mom_dev;           /* dim planes of n_cells */
} fla_psicell_out;

typedef struct {
    uint64_t nonfinite;        /* records with a non-finite n, h or source value */
    uint64_t deposited;        /* droplets that entered a kernel-regression deposit */
    uint64_t droplet_steps;    /* droplet steps integrated by fla_advance (active droplet x step) */
    uint64_t pairs;            /* (cell, droplet) pairs inside the truncated kernels, summed over deposits */
    uint64_t fold_steps;       /* of droplet_steps, those whose J and W were integrated in double precision */
    uint32_t flags;            /* FLA_STATUS_* bits: a bounded device-side wait that ran out */
    uint32_t pad;
} fla_device_status;

/* fla_device_status.flags.  A device-side wait that runs out (about a second)
 * sets its bit and returns; the output of the call it belongs to is not valid,
 * the context stays usable, and fla_sync_status returns FLA_ERR_TIMEOUT. */
#define FLA_STATUS_MLP_TIMEOUT 1u  /* the tensor-core MLP's mbarrier wait */
#define FLA_STATUS_WAIT_TIMEOUT 2u /* a look-back wait of the cell binning (inter-CTA) */

/* Phases of the path, for fla_profile_read. */
enum {
    FLA_PHASE_CARRIER = 0,     /* carrier sampling */
    FLA_PHASE_ADVANCE = 1,     /* fused RK4 advance */
    FLA_PHASE_KEYS = 2,        /* cell keys */
    FLA_PHASE_SORT = 3,        /* radix sort passes */
    FLA_PHASE_BINS = 4,        /* bin starts */
    FLA_PHASE_RECORDS = 5,     /* kernel-regression records */
    FLA_PHASE_GATHER = 6,      /* kernel-regression gather */
    FLA_PHASE_PSICELL = 7,     /* PSI-CELL records and per-cell sums */
    FLA_PHASE_COUNT = 8
};

/* ------------------------------------------------------------------ */

/* Create a context on CUDA device `device` (it also becomes the current
 * device of the calling thread).  Allocates a 64-byte status block.
 * Returns FLA_ERR_CUDA when no usable device exists. */
int fla_create(fla_ctx** out, int device);
void fla_destroy(fla_ctx* ctx);
const char* fla_status_string(int code);
int fla_abi_version(void);

/* Number of value planes of a cloud and the offsets (in values) of x, v, J,
 * W and acc in the flattened per-droplet vector (J and W are -1 for LPT). */
int fla_state_layout(int32_t kind, int32_t dim, int32_t* n_planes, int32_t* off_x, int32_t* off_v,
                     int32_t* off_J, int32_t* off_W, int32_t* off_acc);

/* Bytes of a node array for fla_carrier_sample: (n+1)^dim nodes, each holding
 * u (dim values) then grad u (dim*dim, row-major, G_ij = du_i/dx_j), padded
 * to 8 values (2D) or 12 values (3D).  FLA_F32X2: two arrays of the FLA_F32
 * layout, a then b (each value is a + b), then a 256-byte tail that
 * fla_carrier_sample uses for the components' largest magnitudes. */
size_t fla_carrier_nodes_bytes(const fla_mesh* mesh, int32_t dtype);

/* Sample the analytic carrier and its gradient at time t on the mesh nodes
 * (Eq. 3 needs u at the droplet, Eq. 8 grad u; both are interpolated from
 * these nodes by fla_advance).  nodes_dev: fla_carrier_nodes_bytes bytes,
 * 16-byte aligned.  FLA_F32X2 evaluates the carrier in double precision and
 * splits each value v into a + b: a is v rounded to a multiple of its
 * component's grid Q = 2^(e - 11), where 2^e exceeds the component's largest
 * magnitude over the nodes (so a has at most 12 significant bits), and b is
 * the nearest float to v - a (|b| <= Q/2 + 2^(e - 25); a + b is within
 * 2^(e - 36) of v).
 * Weights on a coarse grid then multiply a exactly, which keeps the advance's
 * interpolation accurate to about 2^(e - 30) at single-precision cost. */
int fla_carrier_sample(fla_ctx* ctx, const fla_carrier_desc* carrier, const fla_mesh* mesh, double t,
                       int32_t dtype, void* nodes_dev, fla_stream_t stream);

/* Host helper: the step from which a release is inactive because it has nearly
 * evaporated: the first s >= step_start with 1 + delta (s - step_start) dt below
 * max(0.01, 4 dt / St0) (Eq. 4 with r0 = 1); FLA_NO_DEADLINE if delta >= 0. */
int fla_batch_deadline(double St0, double delta, double dt, int32_t step_start, int32_t* step_dead);

#define FLA_ADVANCE_RESET_ACC 1u

/* Advance every droplet through steps [step0, step0 + nsteps) of size dt with
 * the carrier frozen at the given node values (re-sample between calls for an
 * unsteady carrier).  Per step s and droplet:
 *   - a pending seed with step_start == s is released: v = u(x0), and for FLA
 *     J = I and W = grad u(x0) (initial data of Eq. 8);
 *   - an active droplet with s >= step_dead becomes inactive;
 *   - an active droplet adds dt * (mdot, F + mdot v) at the step's first RK
 *     stage to acc (App. B, parcel level a-b; F = m x'' below Eq. 9, m = r^3,
 *     mdot = 1.5 delta r), then takes one classical RK4 step of
 *     x' = v, v' = (u - v)/St (Eq. 3) and, for FLA, J' = W,
 *     W' = (grad u . J - W)/St (Eq. 8), with St = St0 (1 + delta (t - t0)) (Eqs. 4-5);
 *   - a droplet that leaves [0,1]^dim becomes inactive.
 * Single-precision FLA clouds with fold_dev set: at the start of each step a
 * droplet with |det J| < tau_fold (single precision) enters the fold guard
 * and one with |det J| > 4 tau_fold (double, from fold_dev) leaves it; while
 * in it, the J and W part of its RK4 step is computed in double precision from
 * the single-precision stage values of grad u and St (fold_steps counts them).
 * Carrier values are bi/trilinear interpolations of nodes_dev (cell index
 * clamped to the mesh).  FLA_ADVANCE_RESET_ACC zeroes acc before the first step.
 * The cloud and nodes must share the dtype; nodes_dev 16-byte aligned. */
int fla_advance(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const void* nodes_dev,
                int32_t step0, int32_t nsteps, double dt, uint32_t flags, fla_stream_t stream);

/* fla_advance (the RK4 step of Eqs. 3-5 and 8, §2) with a processing order:
 * thread t of the launch advances droplet order_dev[t] (device, n words,
 * 4-byte aligned, caller-owned, read only).  Each droplet's arithmetic does not depend on the order, so the
 * results are bit for bit those of fla_advance; the order only decides which
 * droplets share a warp.  With the cell-sorted permutation of the cloud's last
 * binning (fla_workspace_order) the droplets of a warp lie in neighbouring
 * cells and read the same carrier nodes, and the active ones are packed
 * together.  order_dev must be a permutation of [0, n): entries >= n are
 * skipped (those threads advance nothing), repeated entries race.  NULL
 * gives fla_advance. */
int fla_advance_ordered(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const void* nodes_dev,
                        const uint32_t* order_dev, int32_t step0, int32_t nsteps, double dt, uint32_t flags,
                        fla_stream_t stream);

/* Workspace bytes needed by fla_cell_bins, fla_deposit_sources and
 * psicell_deposit for a cloud of n_droplets on this mesh (the maximum over the
 * three, for the given dtype and kernel).  The workspace must be 256-byte
 * aligned. */
int fla_workspace_size(const fla_mesh* mesh, int32_t dtype, int32_t kernel, int64_t n_droplets, size_t* bytes);

/* (No counterpart in the paper: the cell list is this library's.)  Byte
 * offset, within a deposit workspace, of the sorted permutation (n
 * uint32 words: the droplet index at each position of the stable sort by cell
 * key, inactive droplets last) that fla_cell_bins, fla_deposit_sources,
 * psicell_deposit, cic_deposit and fla_learn_grad leave there for a cloud of
 * n_droplets (>= 1) on this mesh.  It stays valid until the workspace serves
 * another cloud; it is the processing order fla_advance_ordered wants. */
int fla_workspace_order(const fla_mesh* mesh, int64_t n_droplets, size_t* offset);

/* Cell binning of a cloud: key_i = linear index of the cell holding x_i
 * (floor(x N) per axis in the cloud's precision, clamped to N-1 so x = 1 is in
 * the last cell), droplets that are not active or lie outside [0,1]^dim get
 * the key n_cells.  Outputs (device, caller-owned): keys_sorted_dev[n] (the
 * keys in stable ascending order, inactive last, with n_cells as key),
 * perm_dev[n] (droplet index at each sorted position; ties keep index order)
 * and bin_start_dev[n_cells + 1] (first sorted position of each cell;
 * bin_start[n_cells] = number of binned droplets).  Bit-exact, deterministic. */
int fla_cell_bins(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, uint32_t* keys_sorted_dev,
                  uint32_t* perm_dev, uint32_t* bin_start_dev, void* workspace_dev, size_t workspace_bytes,
                  fla_stream_t stream);

/* Kernel-regression (Nadaraya-Watson) source terms of an FLA cloud at every
 * cell centre x_c (Eqs. 13 and 16, signs of Eq. 9, App. B cloud level):
 *   n_i = n0/max(|det J_i|, 1e-12) (Eq. 6),  a_i = n_i acc_i / window_dt,
 *   K_i(x_c) = pref_i exp(-q/2) if q <= 9 else 0 (Eq. 14, truncated at 3 sigma),
 *     ISO:   q = |x_c - x_i|^2 / h_i^2, h_i = clamp(h0 |det J_i|^p, h_min, h_max), pref = 1/h_i
 *     ANISO: q = d^T Sigma_i^-1 d, Sigma_i = f h0^2 J J^T + h_min^2 I with
 *            f = min(1, (h_max^2 - dim h_min^2)/tr(h0^2 J J^T)), pref = det(Sigma_i)^-1/2
 *   D_c = sum_i K_i(x_c),  S_mass = -sum K_i a_mass,i / D_c,  S_mom = -sum K_i a_mom,i / D_c,
 *   S = 0 where D_c = 0; times the cell volume when cfg->per_cell.
 * Sums run in a fixed order with compensated (Neumaier) accumulation; the
 * result does not depend on launch timing.  Single precision decides the
 * truncation test on single-precision operands. */
int fla_deposit_sources(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const fla_deposit_cfg* cfg,
                        const fla_sources* out, void* workspace_dev, size_t workspace_bytes,
                        fla_stream_t stream);

/* PSI-CELL box-count sources of a parcel cloud (Eqs. 10-11): for each cell,
 * counts = number of active parcels inside, and
 *   S_mass = -(1/V) sum w_b acc_mass,i / window_dt,  S_mom = -(1/V) sum w_b acc_mom,i / window_dt
 * over those parcels, w_b = batches[b].n0 the real droplets per parcel,
 * V the cell volume (dropped when per_cell).  Counts are exact; sums are in a
 * fixed order. */
int psicell_deposit(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, double window_dt,
                    int32_t per_cell, const fla_psicell_out* out, void* workspace_dev, size_t workspace_bytes,
                    fla_stream_t stream);

/* Cloud-In-Cell sources of a parcel cloud, the C^1 alternative to PSI-CELL
 * that Sec. 1 of the paper names (parcel quantities interpolated linearly to
 * the corners of the occupied cell).  With cell-centred sources the corners
 * are the cell centres around the parcel: each active parcel inside [0,1]^dim
 * gives the cell centred at x_c the weight
 *   W = prod_a max(0, 1 - |x_a - x_c,a| N)
 * (the overlap of a cell-sized cloud around the parcel with that cell), and
 *   S_mass = -(1/V) sum W w_b acc_mass,i / window_dt,  S_mom likewise,
 * over the parcels of the 3^dim cells around each cell; weight that falls on
 * centres outside the mesh is dropped.  counts = parcels whose cell key is the
 * cell (the box count of psicell_deposit).  Same arguments, outputs and
 * workspace as psicell_deposit; the sums run in a fixed order (deterministic,
 * no float atomics). */
int cic_deposit(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, double window_dt, int32_t per_cell,
                const fla_psicell_out* out, void* workspace_dev, size_t workspace_bytes, fla_stream_t stream);

/* ------------------------------------------------------------------------
 * Learned bandwidth correction.  The paper has no counterpart: a small
 * network g corrects each droplet's bandwidth by the factor
 * s = exp(clip(g(f), -2, 2)): for the spherical kernel (Eq. 14 with h of Eq. 15)
 *   h = clamp(h0 |det J|^p * s, h_min, h_max),
 * and for the J-scaled kernel its Lagrangian bandwidth h0 becomes h0 s in
 *   Sigma = f (h0 s)^2 J J^T + h_min^2 I,  f = min(1, (h_max^2 - dim h_min^2) / tr((h0 s)^2 J J^T)),
 * except near fold caustics: for droplets with |det J| < 1e-2 the plain kernel is the fallback
 * (g is evaluated but not applied), because n = n0/|det J| is singular there
 * and a bandwidth learned away from the folds does not transfer to them.  g is
 * 6 -> 64 -> 64 -> 64 -> 1 with SiLU after the hidden layers, evaluated on the
 * tensor cores with BF16 weights and activations and FP32 accumulation (the
 * last layer in FP32 on the CUDA cores).  The features of a droplet are
 *   f0 = ln ||J||_F^2 / 8,  f1 = ln ||cof J||_F^2 / 8 (3D) or ln det(J)^2 / 8 (2D),
 *   f2 = ln |det J| / 8,    f3 = ln n / 8 (n of Eq. 6),
 *   f4 = ln(h0 |det J|^(1/dim) / dx) / 4,  f5 = min(|det J|, 4) / 4,
 * logarithms taken of max(x, 1e-30).
 * Parameters: FLA_MLP_PARAMS FP32 masters W1[64][6], b1[64], W2[64][64],
 * b2[64], W3[64][64], b3[64], W4[64], b4 (rows are output units).
 * ------------------------------------------------------------------------ */
#define FLA_MLP_FEATURES 6
#define FLA_MLP_HIDDEN 64
#define FLA_MLP_PARAMS 8833
#define FLA_MLP_PACKED_BYTES 19472

/* Round the FP32 masters params_dev[FLA_MLP_PARAMS] into the packed device
 * image the tensor-core kernels read (packed_dev, FLA_MLP_PACKED_BYTES,
 * 16-byte aligned, caller-owned).  Re-pack after every parameter update. */
int fla_mlp_pack(fla_ctx* ctx, const float* params_dev, void* packed_dev, fla_stream_t stream);

/* c_i = g(f_i) for n feature rows features_dev[n][6] (FP32; rounded to BF16
 * on the way in) into out_dev[n]. */
int fla_mlp_forward(fla_ctx* ctx, const void* packed_dev, const float* features_dev, int64_t n, float* out_dev,
                    fla_stream_t stream);

/* Training of the learned correction.  For a cloud state and targets T at
 * n_train distinct training cells (T: n_train x (1+dim) FP32, mass then
 * momentum, e.g. the sources of a densely seeded cloud of the same flow), the
 * loss of the learned deposit is
 *   L = 1/(1+dim) sum_k sum_c (S_kc - T_kc)^2 / sum_c T_kc^2,
 * S the sources of fla_deposit_sources with cfg (mlp_dev required).
 * fla_learn_grad runs that deposit into out (dsum_dev required), then adds L
 * to *loss_dev and dL/dtheta (the gradient with respect to the FP32 master
 * parameters, BF16 roundings treated as the identity, the truncation edge held
 * fixed) to grad_dev[FLA_MLP_PARAMS]; callers zero both to start a batch.
 * Single-precision clouds, either kernel (for the J-scaled one the bandwidth
 * moves with g only below the trace cap, f = 1).  workspace: as for
 * fla_deposit_sources; learn_ws: fla_learn_workspace_size bytes, 256-byte
 * aligned.  The sums run in a fixed order: the result is deterministic. */
int fla_learn_workspace_size(fla_ctx* ctx, const fla_mesh* mesh, int64_t n_droplets, size_t* bytes);
int fla_learn_grad(fla_ctx* ctx, const fla_cloud* cloud, const fla_mesh* mesh, const fla_deposit_cfg* cfg,
                   const uint32_t* cells_dev, int64_t n_train, const float* targets_dev, const fla_sources* out,
                   float* grad_dev, float* loss_dev, void* workspace_dev, size_t workspace_bytes, void* learn_ws_dev,
                   size_t learn_ws_bytes, fla_stream_t stream);

/* One Adam step (bias-corrected, step >= 1) on n FP32 parameters:
 *   m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
 *   p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
int fla_adam_step(fla_ctx* ctx, float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int64_t n,
                  float lr, float beta1, float beta2, float eps, int32_t step, fla_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched clouds.  Many single-precision FLA clouds of different sizes,
 * meshes (2D or 3D), carriers and kernels advance and deposit together: each
 * window (window_steps steps of dt) samples every carrier at the window's
 * start, advances every cloud with its window sums reset, and deposits every
 * cloud's kernel-regression sources into its own outputs -- per window a few
 * launches for all clouds instead of a dozen per cloud.  The clouds share one
 * global cell space, so one key pass and one radix sort bin all of them; each
 * cloud's results are those of fla_carrier_sample + fla_advance +
 * fla_deposit_sources for it alone (the advance bit for bit; the deposit with
 * the tile gather that those calls use for 3D, FP64 and anisotropic clouds).
 * The window start step lives on the device (fla_batch_set_step), so
 * fla_batch_run captures its windows once into a CUDA graph and replays it.
 * The first fla_batch_run tunes the launch shapes (advance block size,
 * persistent gather CTAs per SM, gather tile order) on its first windows,
 * timing them with events (it synchronises the stream); none of these
 * changes any result.  The caller owns every buffer; the plan's tables live in
 * the workspace (fla_batch_workspace_size bytes, 256-byte aligned), and the
 * items' buffers must stay valid for the plan's life.
 * ------------------------------------------------------------------------ */
typedef struct fla_batch_plan fla_batch_plan;

typedef struct {
    fla_cloud cloud;           /* FLA_CLOUD_FLA, FLA_F32, no fold guard */
    fla_mesh mesh;
    fla_carrier_desc carrier;  /* sampled at t = step * dt at each window start */
    void* nodes_dev;           /* fla_carrier_nodes_bytes(&mesh, FLA_F32) bytes, 16-byte aligned */
    fla_deposit_cfg cfg;       /* without the learned correction */
    fla_sources out;           /* FP32 outputs on this cloud's mesh */
} fla_batch_item;

int fla_batch_workspace_size(const fla_batch_item* items, int32_t n_items, size_t* bytes);
/* Validates the items, writes the tables into the workspace (synchronous
 * copies) and sets the device step to step0. */
int fla_batch_create(fla_ctx* ctx, const fla_batch_item* items, int32_t n_items, double dt, int32_t window_steps,
                     int32_t step0, void* workspace_dev, size_t workspace_bytes, fla_batch_plan** out);
/* Runs n_windows windows from the device step on stream (a stream other than
 * the legacy default stream for the graph; on the legacy stream, or inside the
 * caller's own capture, the windows are plain launches). */
int fla_batch_run(fla_ctx* ctx, fla_batch_plan* plan, int32_t n_windows, fla_stream_t stream);
int fla_batch_set_step(fla_batch_plan* plan, int32_t step, fla_stream_t stream);
/* The launch shapes in use and the kernel launches per window; returns
 * FLA_ERR_UNSUPPORTED (values still written) before the tuning has run. */
int fla_batch_tuning(const fla_batch_plan* plan, int32_t* advance_threads, int32_t* gather_ctas_per_sm,
                     int32_t* tile_order, int32_t* launches_per_window);
/* Fixes the launch shapes (advance 64/128/256, gather CTAs per SM 1..8, tile
 * order 0 natural / 1 interleaved) and skips the tuning. */
int fla_batch_set_tuning(fla_batch_plan* plan, int32_t advance_threads, int32_t gather_ctas_per_sm,
                         int32_t tile_order);
/* How a window runs.  FLA_BATCH_LAUNCHES: one kernel per phase and group
 * (carrier, advance per dimension, binning, records and gather plan, items
 * and combine per group, step), about 14 per window.  FLA_BATCH_PERSISTENT:
 * one cooperative kernel per window (a memset of its barrier words before
 * it) that runs the same phases, compiled from the same sources, separated
 * by grid barriers; every CTA of the grid is resident, and a barrier wait
 * gives up after about a second (FLA_STATUS_WAIT_TIMEOUT, fla_sync_status
 * returns FLA_ERR_TIMEOUT, the window's outputs are then not valid).  Both
 * give the same results bit for bit.  FLA_BATCH_AUTO (the default): the
 * first fla_batch_run of at least five windows times its fourth window as
 * the persistent kernel and its fifth as launches and keeps the faster
 * (fewer windows: launches).  Changing the mode drops the plan's graph.
 * FLA_ERR_UNSUPPORTED for FLA_BATCH_PERSISTENT where the kernel cannot run
 * (no CTA of it fits an SM). */
enum { FLA_BATCH_AUTO = 0, FLA_BATCH_LAUNCHES = 1, FLA_BATCH_PERSISTENT = 2 };
int fla_batch_set_mode(fla_batch_plan* plan, int32_t mode);
/* The mode in use (FLA_BATCH_AUTO until the first run has chosen) and the
 * tuner's window times in ms (persistent, launches; 0 when not timed). */
int fla_batch_mode(const fla_batch_plan* plan, int32_t* mode, float* persistent_ms, float* launches_ms);
void fla_batch_destroy(fla_batch_plan* plan);

/* Read the device status block (synchronises `stream`); reset != 0 zeroes it
 * afterwards.  Returns FLA_ERR_TIMEOUT when a FLA_STATUS_* timeout bit is set,
 * else FLA_ERR_NONFINITE when nonfinite > 0, else FLA_OK. */
int fla_sync_status(fla_ctx* ctx, fla_stream_t stream, fla_device_status* out, int reset);

/* Allocation-free cell binning, for callers that cannot allocate device
 * memory.  The paper has no counterpart: this exists for host programs that
 * can pass device pointers to buffers they already own but cannot create new
 * ones, such as a solver's C or Fortran coupling layer without a CUDA
 * allocator, or code where cudaMalloc is not allowed because it synchronises
 * the device or because another framework has reserved the memory.
 *
 * Same inputs, outputs and results as fla_cell_bins (bit for bit), but the
 * scratch space is a fixed array compiled into the library (about 5.3 MB of
 * device memory on every GPU that loads the library, held until the process
 * exits) and no fla_ctx is needed.  The call allocates nothing.
 *  - Clouds of more than FLA_NOALLOC_MAX_DROPLETS droplets are rejected with
 *    FLA_ERR_WORKSPACE before anything is enqueued.
 *  - The first call on a device, with that device current, looks up the
 *    array's device address (cudaGetSymbolAddress); make that first call
 *    before any stream capture on that device.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents; nothing in it needs to start at zero.  Calls whose GPU work
 *    overlaps (different streams or host threads without ordering) race on
 *    it and must be serialised by the caller.
 *  - The looked-up address is kept for the life of the process: a host
 *    program that calls cudaDeviceReset between two calls on a device is not
 *    supported (the reset unloads the library's device code and the array).
 *  - Arguments are checked exactly as by fla_cell_bins. */
#define FLA_NOALLOC_MAX_DROPLETS 262144
int fla_cell_bins_noalloc(const fla_cloud* cloud, const fla_mesh* mesh, uint32_t* keys_sorted_dev,
                          uint32_t* perm_dev, uint32_t* bin_start_dev, fla_stream_t stream);

/* Per-phase profiling.  The context always counts the kernels it launches per
 * phase (also while a stream is being captured into a CUDA graph).  With
 * timing enabled it also brackets every phase of every call with CUDA events
 * on the call's stream; fla_profile_read waits for those events and returns,
 * per phase, the summed milliseconds, kernel launches and calls since the last
 * reset.  Timing must stay disabled while a stream is being captured.
 * enable: 0 off, 1 on; reset != 0 zeroes the counters and drops pending events. */
int fla_profile_enable(fla_ctx* ctx, int enable, int reset);
int fla_profile_read(fla_ctx* ctx, int32_t n_phases, double* ms, int64_t* launches, int64_t* calls);
const char* fla_phase_name(int32_t phase);

/* ------------------------------------------------------------------------
 * Two-way coupling: the carrier flow the droplets act on (App. B, carrier
 * level: S_Mom added to Eq. 1, S_Mass to Eq. 2), on a periodic unit square of
 * n x n cells, double precision.  Eq. 1 in vorticity-streamfunction form:
 * omega at the mesh nodes (i h, j h), h = 1/n, psi from the 5-point
 * Laplacian (solved in Fourier space), u = U_x + D_y psi, v = U_y - D_x psi
 * by central differences, U the mean flow; a step of dt advances omega with
 * explicit advection and source curl (from the cell-centred S_Mom) and
 * implicit viscosity nu = 1/Re, and U by dt mean(S_Mom).  Eq. 2 at the cell
 * centres: first-order upwind fluxes through faces whose velocities come from
 * psi at their corner nodes (divergence-free cell by cell), explicit
 * diffusion (read with the physical sign: Eq. 2 prints D grad^2 rho on the
 * left), the mass source.  Node values for fla_advance: u, v and grad u at
 * the (n+1)^2 mesh nodes (node n repeats node 0), grad u by central
 * differences of the nodal velocity.  The state lives in the caller's
 * workspace (fla_ns_workspace_size bytes, 256-byte aligned); all calls are
 * asynchronous on stream except fla_ns_fields with mean_u.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;       /* cells (and nodes) per axis: a power of two, 8..1024 */
    double nu;       /* kinematic viscosity 1/Re (Eq. 1), >= 0 */
    double diff;     /* vapour diffusivity D (Eq. 2), >= 0, with diff dt n^2 <= 1/4 */
    double dt;       /* carrier step */
    /* Optional immersed cylinder (the paper's test case, Sec. 5) by volume
     * penalisation: the momentum equation gains -chi u / eta with
     * chi = (1 - tanh((r - R) n))/2 at the nodes, r the distance to (xc, yc);
     * a fringe strip fringe_x0 <= x <= fringe_x1 relaxes the vorticity at the
     * rate fringe_sigma sin^2(pi (x - x0)/(x1 - x0)), so the periodic wake does
     * not re-enter; hold_mean_flow != 0 keeps the mean flow fixed (a constant
     * inflow), else the mean penalisation force decelerates it.  body = 0: none. */
    int32_t body;
    int32_t hold_mean_flow;
    double body_xc, body_yc, body_r, body_eta;   /* eta > 0, dt / eta <= 1 */
    double fringe_x0, fringe_x1, fringe_sigma;   /* sigma dt <= 1 */
} fla_ns_cfg;

/* Workspace bytes for cfg (0 when cfg is invalid). */
size_t fla_ns_workspace_size(const fla_ns_cfg* cfg);
/* Initial state: omega_dev the nodal vorticity (n*n doubles, x fastest; its
 * mean is dropped), mean_u the mean velocity (host, 2 doubles), rho_dev the
 * vapour at the cells (n*n doubles) or NULL for zero. */
int fla_ns_init(fla_ctx* ctx, const fla_ns_cfg* cfg, const double* omega_dev, const double* mean_u,
                const double* rho_dev, void* workspace_dev, size_t workspace_bytes, fla_stream_t stream);
/* nsub steps of cfg->dt with the droplets' sources held fixed: s_mass_dev
 * (n*n) and s_mom_dev (2 x n*n, component-major), per unit volume, as
 * fla_deposit_sources writes them (src_dtype FLA_F32 or FLA_F64); either may
 * be NULL (no source).  Stable while dt |u| < h (upwind vapour). */
int fla_ns_step(fla_ctx* ctx, const fla_ns_cfg* cfg, const void* s_mass_dev, const void* s_mom_dev,
                int32_t src_dtype, int32_t nsub, void* workspace_dev, size_t workspace_bytes, fla_stream_t stream);
/* The carrier node array for fla_advance (fla_carrier_nodes_bytes of a 2D
 * mesh of n cells; dtype FLA_F32 or FLA_F64, the cloud's). */
int fla_ns_nodes(fla_ctx* ctx, const fla_ns_cfg* cfg, int32_t dtype, void* nodes_dev, void* workspace_dev,
                 size_t workspace_bytes, fla_stream_t stream);
/* The force of the fluid on the cylinder, sum over the nodes of chi u / eta h^2
 * (host, 2 doubles; synchronises stream).  FLA_ERR_ARG without a body. */
int fla_ns_body_force(fla_ctx* ctx, const fla_ns_cfg* cfg, double* force, void* workspace_dev,
                      size_t workspace_bytes, fla_stream_t stream);
/* Read back the nodal vorticity (-Lap_h psi), psi and the vapour (n*n doubles
 * each, any may be NULL) and the mean velocity (host, synchronises stream). */
int fla_ns_fields(fla_ctx* ctx, const fla_ns_cfg* cfg, double* omega_dev, double* psi_dev, double* rho_dev,
                  double* mean_u, void* workspace_dev, size_t workspace_bytes, fla_stream_t stream);

/* Test hook for the bounded device-side waits (no paper passage: the waits
 * are this library's).  what = FLA_STALL_BINNING makes the next binning of this
 * context (fla_cell_bins, a deposit or a parcel deposit) keep one CTA from
 * arriving at its first grid barrier; FLA_STALL_BATCH_WINDOW does the same
 * for the first barrier of the next persistent batch window issued on this
 * context.  The other CTAs wait until their limit (about a second) runs out,
 * then set the abort word and FLA_STATUS_WAIT_TIMEOUT and return, and so does
 * the stalled CTA: the call's output is not valid, fla_sync_status returns
 * FLA_ERR_TIMEOUT, and the context stays usable.  Each bit acts once and
 * clears itself.  FLA_ERR_ARG for unknown bits. */
#define FLA_STALL_BINNING 1u
#define FLA_STALL_BATCH_WINDOW 2u
int fla_test_stall(fla_ctx* ctx, uint32_t what);

#ifdef __cplusplus
}
#endif
#endif /* FLA_H */
