/*
 * nnp.h -- C ABI of the GB300 (sm_103a) neural-network-potential library.
 *
 * The library evaluates an ANI-style neural-network potential (arXiv
 * 2207.14276, Sec. "Neural Network Potentials", Eqs. 2-5) and its analytic
 * forces on one GPU:
 *   cell-list neighbour search under a cutoff  ->  atomic environment vectors
 *   (radial Gaussian shells, Eq. 4, and angular triplet terms, Eq. 5, with the
 *   cosine cutoff of Eq. 3; one radial block per species and one angular block
 *   per unordered species pair)  ->  one feed-forward network per species,
 *   summed to the energy (Eq. 2)  ->  analytic backward to per-atom forces.
 * The hybrid model of Eq. 7 is supported through a per-atom mask: only masked
 * atoms (the solute region P) are centres or neighbours, which yields V_ML(P).
 *
 * As in the paper's engine interface (Sec. "A General Machine Learning
 * Platform": positions in, energies and forces out, device pointers handed
 * over without copies), inputs and outputs are caller-owned DEVICE pointers
 * and every compute call is asynchronous on the caller's CUDA stream.  Only
 * nnp_energy_forces_host takes host buffers.
 *
 * Units: Angstrom, kcal/mol, kcal/mol/Angstrom.
 *
 * Errors: every call returns an NNP_* status code and never aborts;
 * nnp_last_error() gives a thread-local message for the last failure.
 * Conditions that only the device can see (a species index out of range, a
 * non-finite coordinate, a neighbour list over capacity) are recorded in a
 * device status word of the handle and reported by nnp_sync_status().
 *
 * Concurrency: a handle owns one work arena.  Calls on one handle must be
 * ordered on one stream (or otherwise serialised by the caller); to overlap
 * work on two streams use two handles (nnp_clone shares the weights).
 */
#ifndef NNP_H
#define NNP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
  NNP_OK = 0,
  NNP_ERR_ARG = 1,            /* bad argument (null pointer, negative size, ...)      */
  NNP_ERR_SPECIES = 2,        /* a species index >= n_species (device-detected)       */
  NNP_ERR_BOX_TOO_SMALL = 3,  /* periodic edge < 2 * max cutoff (minimum image fails)  */
  NNP_ERR_NONFINITE = 4,      /* NaN/Inf coordinate in the ML region (device-detected) */
  NNP_ERR_CAPACITY = 5,       /* neighbour list over capacity; capacity has been grown,
                                 repeat the call                                       */
  NNP_ERR_OOM = 6,            /* device allocation failed / over the HBM budget        */
  NNP_ERR_CUDA = 7,           /* a CUDA runtime call failed                            */
  NNP_ERR_TIMEOUT = 8,        /* a bounded device-side wait gave up                    */
  NNP_PENDING = 9,            /* result not ready yet                                  */
  NNP_ERR_UNSUPPORTED = 10,   /* hyper-parameters outside what the kernels implement   */
  NNP_ERR_BOUNDS = 11         /* bounds-checked build only: a kernel found an index out
                                 of range, skipped the access and recorded the site     */
};

/* precision of the per-species networks (AEVs, their backward and the forces
 * are FP32 in every mode; energies and virials are reduced in FP64) */
enum {
  NNP_FP32 = 0,       /* FP32-accurate networks on the fastest such path, which
                         on this GPU is NNP_FP32_SPLIT                             */
  NNP_BF16_MLP = 1,   /* network layers on tcgen05 tensor cores, BF16 operands and
                         FP32 accumulation                                         */
  NNP_FP32_SPLIT = 2, /* network layers on tcgen05 tensor cores with every FP32
                         operand split into two BF16 parts, x = hi + lo, and the
                         three products hi*hi + lo*hi + hi*lo accumulated in FP32
                         (the "bf16x3" scheme of Henry, Tang and Heinecke, ARITH
                         2019): about 16 significant bits per operand           */
  NNP_FP32_SIMT = 3   /* network layers in FP32 on the FMA pipes                  */
};

typedef struct nnp_handle nnp_handle;

/* Species handled by the model; index order is the AEV block order (the paper's
 * ANI models: H,C,N,O and, for ANI-2x, S,F,Cl).  n_species <= 8. */
typedef struct {
  int n_species;
  int atomic_numbers[8];
} nnp_species_t;

/* AEV hyper-parameters (Eqs. 3-5).  rc_r / rc_a: radial / angular cutoff radii;
 * eta_r, shf_r[]: radial Gaussian width and centres; eta_a, shf_a[]: Gaussian of
 * the averaged distance in the angular term; zeta and shf_z[] (theta_s values, in
 * radians): angular factor (1 + cos(theta - theta_s))^zeta with the 2^(1-zeta)
 * prefactor; theta = acos(cos_scale * cos_angle) (cos_scale = 1 is the paper's
 * form).  The kernels implement n_shf_r = 16, n_shf_a = 4, n_shf_z = 8 and an
 * integer zeta in [1, 64]; anything else returns NNP_ERR_UNSUPPORTED. */
typedef struct {
  float rc_r, eta_r;
  int n_shf_r;
  float shf_r[32];
  float rc_a, eta_a, zeta;
  int n_shf_a;
  float shf_a[16];
  int n_shf_z;
  float shf_z[16];
  float cos_scale;
} nnp_aev_params_t;

/* Per-species feed-forward networks (Eq. 2; one per species and ensemble member,
 * CELU activations between layers, linear output of width 1).
 * widths[0] must equal the AEV length S*n_shf_r + S(S+1)/2*n_shf_a*n_shf_z and
 * widths[n_layers] must be 1; n_layers = 4 is implemented.
 * params: host FP32, flat, copied at nnp_create:
 *   for e < n_ensemble, for s < n_species, for l < n_layers:
 *       W_l row-major [widths[l+1], widths[l]], then b_l [widths[l+1]]
 * species_shift: host [n_species] energy added per atom (NULL = zeros).
 * The ensemble energy is the arithmetic mean of the members. */
typedef struct {
  int n_ensemble;
  int n_layers;
  const int* widths;
  const float* params;
  const double* species_shift;
  float celu_alpha;
} nnp_weights_t;

/* One system of a batched call.  All pointers are device pointers owned by the
 * caller.  coords [n_atoms,3] float32; species [n_atoms] uint8 (< n_species);
 * mask [n_atoms] uint8, 1 = atom is in the ML region, NULL = all atoms;
 * periodic != 0: orthorhombic box of edges box[3] with the minimum-image
 * convention (each edge >= 2 * max(rc_r, rc_a)); otherwise box is ignored.
 * Outputs: energy (1 double, written), forces [n_atoms,3] (written; zero for
 * atoms outside the mask; NULL = not computed), virial [9] row-major
 * -sum_edges u (x) dE/du (NULL = not computed), atom_energies [n_atoms] float
 * (NULL = not written; zero outside the mask).  When no system of a call asks
 * for forces or a virial, the backward kernels are skipped (energy-only
 * re-evaluation, e.g. of stored snapshots for reweighting). */
typedef struct {
  int64_t n_atoms;
  const float* coords;
  const uint8_t* species;
  const uint8_t* mask;
  double box[3];
  int periodic;
  double* energy;
  float* forces;
  double* virial;
  float* atom_energies;
} nnp_system_t;

/* Create a model.  Copies the parameters to the device (weights are owned by the
 * library).  hbm_budget_bytes bounds the work arena (0 = no bound); the arena is
 * grown on demand in proportion to the number of atoms, as in the paper's
 * bounded upfront buffer (Sec. "Massive Parallelism within Tinker-HP").
 * precision: one of the NNP_FP32* modes or NNP_BF16_MLP (enum above).  On
 * success *out holds the handle. */
int nnp_create(const nnp_species_t* species, const nnp_aev_params_t* aev,
               const nnp_weights_t* weights, int precision, size_t hbm_budget_bytes,
               nnp_handle** out);

/* A second handle on the same device weights with its own work arena, for
 * overlapping calls on another stream.  Destroy each handle separately. */
int nnp_clone(const nnp_handle* h, nnp_handle** out);

void nnp_destroy(nnp_handle* h);

/* Pre-size the work arena for up to max_atoms atoms in one call (all systems of
 * a batch together), max_systems systems per batch and the given neighbour
 * capacities per atom (0 keeps the current value; at most 512 radial neighbours
 * per atom are supported, more returns NNP_ERR_UNSUPPORTED).  Synchronises the device.
 * Calls that stay within the reservation allocate nothing. */
int nnp_reserve(nnp_handle* h, int64_t max_atoms, int max_systems, int max_neighbors_radial,
                int max_neighbors_angular);

/* Energy and forces of one system (Eqs. 2-5; Eq. 7 with a mask), asynchronous on
 * `stream` (a cudaStream_t, NULL = legacy default stream).
 *   coords   device float32 [n_atoms,3]
 *   species  device uint8 [n_atoms]
 *   box_host host double[3] orthorhombic edges, NULL = non-periodic
 *   mask     device uint8 [n_atoms] or NULL
 *   energy   device double[1]; forces device float32 [n_atoms,3] or NULL
 *            (energy only);
 *   virial   device double[9] or NULL
 * Returns NNP_OK once the work is enqueued; device-side failures are read with
 * nnp_sync_status. */
int nnp_energy_forces(nnp_handle* h, int64_t n_atoms, const float* coords,
                      const uint8_t* species, const double* box_host, const uint8_t* mask,
                      double* energy, float* forces, double* virial, void* stream);

/* Batched evaluation of n_sys independent systems (molecules, replicas, lambda
 * windows) in one pass: all systems' atoms share the neighbour, AEV and network
 * kernels, so small systems fill the GPU together.  `systems` is a HOST array of
 * descriptors holding device pointers.  Asynchronous like nnp_energy_forces. */
int nnp_energy_forces_batch(nnp_handle* h, int n_sys, const nnp_system_t* systems,
                            void* stream);

/* End-to-end convenience for host callers: host buffers in and out, copies to
 * and from the device inside, synchronous.  coords_h [n,3] float32, species_h
 * [n] uint8, mask_h [n] or NULL, box_host double[3] or NULL; energy_h double[1],
 * forces_h float32 [n,3], virial_h double[9] or NULL.  Copies, evaluation and
 * the status read run on the legacy default stream with one synchronisation;
 * page-locked buffers keep the copies asynchronous.  energy_h and virial_h are
 * written only when the call returns NNP_OK; forces_h may hold partial results
 * after an error.  Retries once after a capacity overflow. */
int nnp_energy_forces_host(nnp_handle* h, int64_t n_atoms, const float* coords_h,
                           const uint8_t* species_h, const double* box_host,
                           const uint8_t* mask_h, double* energy_h, float* forces_h,
                           double* virial_h);

/* ---------------------------------------------------------------- differentiation
 * Vector-Jacobian product of (E, F) for training by force matching: given
 * gE = dL/dE and v = dL/dF of a loss L(E, F) (e.g. sum (F - F_target)^2, where
 * v = 2 (F - F_target)), returns
 *   dL/dcoords  = -gE F + (d/de) F(r + e v)      (a Hessian-vector product), and
 *   dL/dweights = gE dE/dweights - d/dweights [ sum_i dE/dG_i . J_i v ],
 * the second derivatives of Eqs. 2-5 taken analytically: the AEV Jacobian along
 * v, a forward-over-reverse pass through the networks, and the AEV backward
 * in dual-number arithmetic.  FP32 handles only.  The call recomputes the
 * forward pass and also writes E and F.
 * dL_dweights: device float [nnp_n_weights(h)], flat in the nnp_weights_t layout,
 * written (summed over the systems of a batch).  Per system: dL_dF device float
 * [n,3] (input), dL_dcoords device float [n,3] (output; zero outside the mask).
 * Asynchronous on `stream`. */
typedef struct {
  nnp_system_t sys;      /* inputs and the energy/forces outputs (virial ignored) */
  double dL_dE;
  const float* dL_dF;
  float* dL_dcoords;
} nnp_vjp_system_t;

int nnp_force_vjp_batch(nnp_handle* h, int n_sys, const nnp_vjp_system_t* systems,
                        float* dL_dweights, void* stream);
int nnp_force_vjp(nnp_handle* h, int64_t n_atoms, const float* coords, const uint8_t* species,
                  const double* box_host, const uint8_t* mask, double dL_dE,
                  const float* dL_dF, double* energy, float* forces, float* dL_dcoords,
                  float* dL_dweights, void* stream);
/* Number of network parameters (length of the flat weight vector). */
int64_t nnp_n_weights(const nnp_handle* h);

/* ---------------------------------------------------------------- serving
 * A continuous-batching server for streams of independent energy+force
 * requests (many small molecules, or new solute coordinates for solvated boxes
 * kept resident on the device -- the shape of the free-energy windows and
 * replicas of the paper's hybrid simulations).  The server owns n_lanes lanes;
 * each lane is a clone of `model` (shared weights, own work arena reserved for
 * max_batch_atoms atoms and max_batch_systems systems), its own CUDA stream and
 * a worker thread.  Requests join one FIFO queue; a free lane takes every queued
 * request that fits its reservation (admission by device-memory footprint),
 * stages the inputs with one host-to-device copy, evaluates them in one batched
 * pass and copies the results back.  Lanes run concurrently, so batches overlap
 * on the device, and requests arriving while lanes are busy are admitted as soon
 * as a lane frees.
 *
 * nnp_request_t: HOST buffers owned by the caller, which must stay valid until
 * the request is polled complete.
 *   resident_id < 0: a standalone system of n_atoms atoms (coords [n,3],
 *     species [n], mask [n] or NULL, box/periodic as in nnp_system_t);
 *   resident_id >= 0: the first n_atoms atoms of the registered resident system
 *     get the new coordinates `coords`; species, mask and box are the resident's.
 *   energy: double[1] out; forces: float [n_atoms,3] out (NULL = not returned). */
typedef struct {
  int64_t n_atoms;
  const float* coords;
  const uint8_t* species;
  const uint8_t* mask;
  double box[3];
  int periodic;
  int resident_id;
  double* energy;
  float* forces;
} nnp_request_t;

typedef struct nnp_server nnp_server;

/* Create a server on the current device.  `model` must outlive the server. */
int nnp_server_create(const nnp_handle* model, int n_lanes, int64_t max_batch_atoms,
                      int max_batch_systems, nnp_server** out);
/* Stop the lanes (queued requests are finished first) and free everything. */
void nnp_server_destroy(nnp_server* s);
/* Keep a system resident on the device (host inputs copied once); *resident_id
 * names it in later requests.  Synchronous. */
int nnp_server_register(nnp_server* s, int64_t n_atoms, const float* coords_h,
                        const uint8_t* species_h, const uint8_t* mask_h,
                        const double* box_host, int* resident_id);
/* Queue a request; *ticket identifies it.  Thread-safe.  NNP_ERR_OOM if the
 * request does not fit a lane's reservation. */
int nnp_server_submit(nnp_server* s, const nnp_request_t* request, uint64_t* ticket);
/* NNP_PENDING while the request runs (wait = 0); with wait != 0 blocks until it
 * completes.  On completion returns the request's status, writes the time from
 * submission to completion (seconds) to *latency_s (may be NULL) and forgets
 * the ticket. */
int nnp_server_poll(nnp_server* s, uint64_t ticket, int wait, double* latency_s);
/* Batches and requests completed so far (either pointer may be NULL). */
int nnp_server_stats(nnp_server* s, long long* batches, long long* requests);

/* Synchronise `stream`, read and clear the handle's device status word.  Returns
 * NNP_OK or the first device-detected error since the last check
 * (NNP_ERR_SPECIES, NNP_ERR_NONFINITE, NNP_ERR_CAPACITY, NNP_ERR_TIMEOUT).  After
 * NNP_ERR_CAPACITY the neighbour capacity has already been grown to what the
 * failed call needed, so repeating the call succeeds. */
int nnp_sync_status(nnp_handle* h, void* stream);

/* Length of the atomic environment vector. */
int nnp_aev_dim(const nnp_handle* h);

/* Deterministic mode (off by default): every energy and force call of the handle
 * returns bitwise identical energies, forces and virials for identical inputs.
 * The atoms of each cell are ordered by input index and the AEV rows of each
 * species by packed position (both otherwise follow atomic counters); every
 * force term is written to its own slot (per centre and neighbour-list entry)
 * and a gather sums them in list order, energies and virials are summed over
 * each system's atoms in a fixed order, and the lanes of a warp add into the
 * shared-memory accumulators one after the other.  For catching races: a
 * result that changes between repeated calls in this mode is a bug.  Costs
 * extra memory ((cap_r + cap_a + 1) float4 and 10 doubles per atom) and time.
 * Not covered: the force VJP, and on the FP32 FMA path the ensembles' six-GEMM
 * chain (its output-layer dot products add partial sums atomically; the fused
 * kernel of one-network models is covered).  Takes effect from the next call. */
int nnp_set_deterministic(nnp_handle* h, int enable);

/* ---------------------------------------------------------------- build variants
 * The library also builds as libnnp_debug.so with index checks in its kernels
 * (the neighbour lists' entries and the cells they come from, the packed
 * positions and AEV rows, the force targets and triplet slots of the AEV
 * backward, the GEMM epilogues' output rows).  A failed check skips the access,
 * sets a flag in the handle's status word and records the first failing site;
 * the call then returns NNP_ERR_BOUNDS with the site in nnp_last_error().  It
 * stands in for a memory checker: same API, same results, slower kernels.
 * nnp_build_flags: NNP_BUILD_BOUNDS_CHECKS set in the bounds-checked build. */
#define NNP_BUILD_BOUNDS_CHECKS 1
int nnp_build_flags(void);

/* The check itself, run on the host (for tests of the check's bookkeeping):
 * returns 1 if 0 <= i < n, else ORs 32 into status[0] (status[0..3], caller
 * memory), stores `site` (1..10, as listed above in that order) in status[3] if
 * it holds 0, and returns 0.  Returns -1 (nnp_last_error says why) for a null
 * status or an unknown site. */
int nnp_debug_check_index(int site, int64_t i, int64_t n, int* status);
/* Tensor-core paths (NNP_BF16_MLP, NNP_FP32_SPLIT): enable != 0 runs the layers
 * after the first -- L2, L3 with the output layer, and their backward B3, B2 --
 * as one fused kernel per 128-row tile with the activations in shared memory
 * (widths multiples of 16, at most 256); 0 runs them as four layer GEMMs
 * through HBM.  Both give the same result to rounding order.  Default: off (on
 * the 100k-atom 8-network workload the fused kernel ties with the four GEMMs on
 * the split path and is slower on BF16).  Clones inherit the setting.  No
 * effect on NNP_FP32_SIMT handles. */
int nnp_set_fused_chain(nnp_handle* h, int enable);
/* Tensor-core paths: enable != 0 (the default) writes each AEV row only in the
 * 64-column slices that hold a species or species-pair block with any term
 * (the rest of the row is zero: for a water molecule's atom most of the
 * 7-species blocks), and runs the first layer over the slices that are live in
 * some row of each 128-row tile and the last backward layer only for the
 * columns of those slices; 0 writes and multiplies whole rows.  The result is
 * the same (the skipped products are exact zeros; the dE/dG columns not
 * computed are those the forces never read).  While it is on, nnp_debug_rows
 * returns 0 for AEV slices a row does not hold and for dE/dG slices its tile
 * does not compute. */
int nnp_set_sparse_rows(nnp_handle* h, int enable);
/* The live-slice masks of the last call's 128-row AEV tiles (bit k: columns
 * 64k .. 64k+63), copied to out_host (at most max_tiles); *n_tiles receives the
 * count (0 when the last call wrote whole rows).  Synchronises `stream`. */
int nnp_debug_tile_masks(nnp_handle* h, void* stream, uint32_t* out_host, int max_tiles,
                         int* n_tiles);
/* BF16 handles of one-network models: enable != 0 computes the AEV rows of each
 * 128-row species tile in shared memory and feeds them to the first layer's
 * tensor-core GEMM in the same kernel, so the AEV is never written to HBM (the
 * fused AEV -> first-layer step); 0 (the default) runs the AEV kernel and the
 * layer GEMM.  Same result to rounding order.  While it is on, nnp_debug_rows
 * cannot return AEV rows (NNP_ERR_UNSUPPORTED).  Falls back to the two kernels
 * where the tile and the neighbour staging do not fit in shared memory. */
int nnp_set_fused_aev_l1(nnp_handle* h, int enable);
/* The network path a handle runs: NNP_FP32_SPLIT, NNP_FP32_SIMT or NNP_BF16_MLP
 * (NNP_FP32 resolves to one of the first two at nnp_create); -1 for a null handle. */
int nnp_network_path(const nnp_handle* h);

/* Number of kernels the last compute call enqueued (for launch accounting). */
int nnp_last_launch_count(const nnp_handle* h);

/* Persistent neighbour lists with a Verlet skin (paper Sec. "Neighbour lists":
 * the lists are rebuilt only when atoms have moved far enough, as in the MD
 * engine's multiple-time-step loop).
 *
 * nnp_set_skin(h, skin): skin in [0, 3] A; 0 (the default) rebuilds the cell
 * and neighbour lists on every call.  With skin > 0 the lists of energy/force
 * calls on this handle (nnp_energy_forces, nnp_energy_forces_batch and the host
 * entry point) are built with cutoffs Rc + skin and kept: a later call reuses
 * them when its batch has the same layout (number of systems, atom counts,
 * species and mask pointers, boxes) and no ML atom has moved more than skin/2
 * (minimum image) since the build; the check runs on the device, so calls stay
 * asynchronous.  The AEV kernels drop list entries beyond the true cutoffs, so
 * results equal those of rebuilt lists up to FP32 summation order.  The caller
 * must not change the contents of the species or mask arrays while the lists
 * persist (pass other arrays, or call nnp_set_skin again, to force a rebuild).
 * A force VJP call on the handle rebuilds lists at the cutoffs; the next energy
 * call rebuilds the skin lists.  Returns NNP_OK or NNP_ERR_ARG.
 *
 * nnp_list_stats(h, stream, &builds, &calls): synchronises `stream`; builds =
 * list builds on the device since the skin was set (or the arena last grew),
 * calls = energy/force calls made with a skin. */
int nnp_set_skin(nnp_handle* h, float skin);
int nnp_list_stats(nnp_handle* h, void* stream, int64_t* builds, int64_t* calls);

/* Velocity-Verlet kick and drift for a multiple-time-step driver that evaluates
 * the potential on the ML region every outer step (paper Eq. 7: the hybrid
 * energy V_MM + V_ML(P) - V_MM(P), integrated with RESPA; the MM terms belong to
 * the host engine).  For every atom i with mask == NULL or mask[i] != 0:
 *   v_i += dt_kick_fs * 4.184e-4 * F_i * inv_masses[i]   (F in kcal/mol/A,
 *                                                         masses in g/mol, v in A/fs)
 *   x_i += dt_drift_fs * v_i
 * coords, velocities: device float [n][3], updated in place; forces: device
 * float [n][3] or NULL (no kick); inv_masses: device float [n] (0 freezes an
 * atom); mask: device uint8 [n] or NULL.  kinetic: device double or NULL; when
 * given it receives sum_i m_i |v_i|^2 / 2 in kcal/mol over the masked atoms
 * after the kick.  Asynchronous on `stream`.  Returns NNP_OK, NNP_ERR_ARG or
 * NNP_ERR_CUDA (launch failure). */
int nnp_integrate(int64_t n_atoms, float* coords, float* velocities, const float* forces,
                  const float* inv_masses, const uint8_t* mask, float dt_kick_fs,
                  float dt_drift_fs, double* kinetic, void* stream);

/* Per-stage timing with CUDA events recorded on the caller's stream around the
 * kernels of each stage (prep, neighbors, aev_fwd, mlp_l1 .. mlp_b1, aev_bwd,
 * finalize, mlp_cvt).  nnp_profile(h, 1) enables recording for later calls;
 * nnp_profile_read synchronises the recorded events, adds their durations to
 * per-stage totals and copies up to max_stages totals (milliseconds) and event
 * pair counts into ms_out / calls_out (either may be NULL); *n_stages receives
 * the number of stages; reset != 0 clears the totals afterwards.
 * nnp_profile_stage_name(i) names stage i. */
int nnp_profile(nnp_handle* h, int enable);
int nnp_profile_read(nnp_handle* h, int reset, double* ms_out, long long* calls_out,
                     int max_stages, int* n_stages);
const char* nnp_profile_stage_name(int i);

/* Thread-local description of the last error (empty string if none). */
const char* nnp_last_error(void);

/* ---------------------------------------------------------------- allocation-free call
 * nnp_energy_forces_noalloc: the same evaluation as nnp_energy_forces, for
 * callers that cannot let the library allocate device memory while they run --
 * for example an MD engine that reserves the whole HBM budget for itself up
 * front (an allocation would then fail), or a time loop in which a cudaMalloc
 * or cudaFree would stall the whole device.  The paper has no counterpart of
 * this entry point; it is a deployment aid.
 *
 * Its work buffers live in one file-scope device array of
 * NNP_NOALLOC_SCRATCH_BYTES bytes (32 MiB) that every GPU holds from the moment
 * the library is loaded until the process exits.  The call performs no
 * cudaMalloc, no cudaFree and no allocating library call.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.
 *
 * Limits: one system, FP32 handles only (NNP_ERR_UNSUPPORTED otherwise); the
 * input atoms, their neighbour lists (at most 256 radial and 96 angular
 * neighbours per atom), AEV rows and network buffers must fit in the array:
 * about 6,900 atoms for the 4-species 384-160-128-96-1 network (one-network models
 * keep their activations on chip), fewer for the 7-species model and far fewer
 * for ensembles; nnp_noalloc_max_atoms returns the exact limit of a handle.
 * A larger request returns NNP_ERR_ARG with a message giving the bytes needed
 * and the limit, before any work is enqueued.
 *
 * Every call reuses the same array and overwrites what the previous call left
 * there (the call clears its counters and accumulators itself).  Calls whose
 * GPU work overlaps -- on two streams, from two threads or through two handles
 * -- therefore race and return wrong results; serialise them.
 *
 * Arguments as for nnp_energy_forces.  The call is synchronous: it waits for
 * `stream` and returns NNP_OK or the error the device detected
 * (NNP_ERR_SPECIES, NNP_ERR_NONFINITE, or NNP_ERR_CAPACITY if an atom has more
 * neighbours than the fixed lists hold). */
#define NNP_NOALLOC_SCRATCH_BYTES (32u << 20)
int nnp_energy_forces_noalloc(nnp_handle* h, int64_t n_atoms, const float* coords,
                              const uint8_t* species, const double* box_host,
                              const uint8_t* mask, double* energy, float* forces,
                              double* virial, void* stream);
/* The largest n_atoms nnp_energy_forces_noalloc accepts for this handle's model
 * (0 for a BF16 handle).  Host computation only. */
int nnp_noalloc_max_atoms(const nnp_handle* h, int64_t* max_atoms);

/* ---------------------------------------------------------------- diagnostics
 * Read back intermediate results of the LAST compute call on this handle (for
 * parity tests against a reference implementation).  Asynchronous on `stream`;
 * the handle's arena must not have been reused by a later call.
 *
 * nnp_debug_rows: which = 0 -> atomic environment vectors G_i (Eqs. 4-5),
 *   which = 1 -> dE/dG_i (the network gradient fed to the force kernel).
 *   out: device float32 [n_in_total, aev_dim], row i = input atom i of the
 *   batch (systems concatenated in call order); rows of atoms outside the
 *   mask are left untouched.
 * nnp_debug_neighbors: out: device int32 [n_in_total, cap]; out[i][t] is the
 *   batch input index of the t-th neighbour of atom i (radial cutoff list, or
 *   the angular-cutoff sub-list if angular != 0), -1 past the end; rows of
 *   atoms outside the mask are left untouched. */
int nnp_debug_rows(nnp_handle* h, int which, float* out, void* stream);
/* Exercises the failure path of the bounded device waits: one thread waits on
 * an mbarrier phase that nothing completes, gives up after `limit` polls and
 * records NNP_ERR_TIMEOUT in the handle's status word (read it with
 * nnp_sync_status); the context stays usable. */
int nnp_debug_wait_probe(nnp_handle* h, unsigned limit, void* stream);
int nnp_debug_neighbors(nnp_handle* h, int angular, int cap, int* out, void* stream);
/* The cell grid the neighbour search (Sec. "Massive Parallelism within
 * Tinker-HP": linked cells of edge >= the cutoff) builds for one system whose
 * ML region spans len[3] A (the box edges if periodic), with list cutoff rc A
 * and n_atoms input atoms: nc_out[3] cells per dimension, each cell at least rc
 * wide, and the total (returned in *cells_out) at most 2 n_atoms + 27, the cell
 * capacity the work arena holds per system.  Host computation only (no device
 * call); the kernels use the same function.  NNP_ERR_ARG on null pointers or
 * rc <= 0. */
int nnp_debug_cell_grid(const float* len, float rc, int64_t n_atoms, int* nc_out,
                        int64_t* cells_out);

#ifdef __cplusplus
}
#endif
#endif /* NNP_H */
