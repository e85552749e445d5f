/*
 * lattice.h -- C ABI of the GB300 checkerboard spin-lattice sweep library.
 *
 * Method: Levy, Cohen & Rabani, "Simulating lattice spin models on GPUs"
 * (arXiv:1209.0296).
 *   - §III.A, Eq. 2: 2D Ising model H = -J sum_<ij> s_i s_j, Metropolis
 *     acceptance min[1, exp(-dH/T)], checkerboard (sublattice) parallel
 *     sweep: one colour of sites is updated while the other is held fixed
 *     (algorithm steps 5-8, Fig. 2); extended here with a field h, to 3D,
 *     and to spin-S values (§III: "easily extended to any spin dimension
 *     and value").
 *   - §III.B, Eq. 3: the North-East kinetically constrained model: a site
 *     may change only if its north (upper) and east (right) neighbours are
 *     up; the initial state is up with probability c (the equilibrium
 *     concentration).
 *   - §IV: per-thread random numbers; replaced here by counter-based
 *     Philox4x32-10 (Salmon et al., SC'11) so results do not depend on the
 *     thread mapping: every result is bit-exact with a CPU restatement.
 *
 * Conventions shared by every entry point:
 *   - H = -J sum_<ij> s_i s_j - h sum_i s_i for both models; each bond
 *     (i, i+e_d) is counted once per direction d (so for L = 2 a pair is
 *     counted twice, in H and in dE alike).  The paper's North-East
 *     Hamiltonian with B = +1 corresponds to h = -1 here.
 *   - Sites are stored x fastest: i = x + L*(y + L*z).  colour(i) =
 *     (x+y+z) mod 2.  One sweep = all colour-0 sites, then all colour-1
 *     sites.  Periodic boundaries in every direction; L must be even.
 *   - Spin values (int8): two_S = 1 gives s = +-1; even two_S gives
 *     s in {-S..S}; odd two_S > 1 gives s in {-two_S, -two_S+2, .., two_S}
 *     (twice the half-integer value).
 *   - Randomness: key = (seed lo, seed hi); counter = (g, sweep lo,
 *     sweep hi, colour), g = row * G + (j >> sh), row = y + L*z,
 *     j = x >> 1, G = ceil((L/2) / 2^sh); sh = 2 (4 sites per draw, word
 *     j & 3 decides acceptance) for spin-1/2, sh = 1 (2 sites per draw,
 *     word 2(j&1) decides acceptance, word 2(j&1)+1 picks the proposal) for
 *     two_S > 1.  Initial states use counter (i >> 2, 0, 0, 2), word i & 3.
 *   - Acceptance: dE <= 0 is accepted without a draw; otherwise the move is
 *     accepted iff u < floor(exp(-dE/T) * 2^32), the threshold being
 *     computed on the host in double precision.  North-East with
 *     J = h = 0 reads T_or_c as the concentration c, with
 *     p(down->up) = min(1, c/(1-c)) and p(up->down) = min(1, (1-c)/c).
 *   - Spin-S proposal: k' = (k + 1 + floor(u*two_S / 2^32)) mod (two_S+1),
 *     k the state index (0 = most negative spin).
 *   - Return codes: 0 on success, a negative LAT_E* code on error;
 *     lattice_strerror() names it.  Argument errors are reported before any
 *     GPU work is queued.  Handles are owned by the library and are not
 *     thread-safe; a server handle is.
 *   - Host buffers passed in are owned by the caller; the library never
 *     keeps a pointer to them after the call returns.
 *   - All GPU work of a handle runs on the stream given at creation (NULL =
 *     the legacy default stream).  Entry points that return host data
 *     synchronise that stream.
 */
#ifndef LATTICE_H
#define LATTICE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum lattice_status {
    LAT_OK = 0,
    LAT_EINVAL = -1,   /* invalid argument */
    LAT_ENOMEM = -2,   /* device or host allocation failed */
    LAT_ECUDA = -3,    /* a CUDA call failed (see lattice_last_cuda_error) */
    LAT_ETIMEOUT = -4, /* a bounded device-side wait gave up */
    LAT_EBUSY = -5,    /* result not ready yet (server poll) */
    LAT_ENOTSUP = -6,  /* valid but unsupported combination */
    LAT_ERANGE = -7,   /* index or size out of range */
    LAT_ENOENT = -8    /* unknown id */
};

/* LAT_POTTS: the q-state Potts model, H = -J sum_<ij> delta(s_i, s_j) -
 * h sum_i delta(s_i, 0), with q = two_S + 1 states (2..9) stored as the
 * labels 0..q-1 (the remark closing the paper's §III.A: the method suits the Potts model). */
enum lattice_model { LAT_ISING = 0, LAT_NE = 1, LAT_POTTS = 2 };
enum lattice_init {
    LAT_INIT_COLD = 0,        /* every spin at its top value (+1 for spin-1/2) */
    LAT_INIT_RANDOM = 1,      /* uniform over the 2S+1 values */
    LAT_INIT_EQUILIBRIUM = 2  /* North-East, c-mode: up with probability c (§III.B) */
};
enum lattice_layout {
    LAT_INT8 = 0,      /* one int8 spin per site */
    LAT_BITPACKED = 1  /* spin-1/2, 2D only: one bit per site, colour-separated planes */
};
/* Sweep dynamics for lattice_set_dynamics. */
enum lattice_dynamics {
    LAT_DYNAMICS_CHECKERBOARD = 0, /* colour 0 then colour 1 (§III.A steps 5-8); the default */
    LAT_DYNAMICS_RANDOM_SITE = 1,  /* the paper's random-sub-lattice, random-site algorithm
                                      (§III.B, second algorithm) */
    LAT_DYNAMICS_RANDOM_SITE_BALANCED = 2  /* its balance-preserving variant (§III.B, after
                                              Fig. 5): single-colour rounds */
};
/* Kernel selection for lattice_set_kernel (tests and the autotuner). */
enum lattice_kernel {
    LAT_KERNEL_AUTO = 0,    /* library choice (tuned tile shape when eligible) */
    LAT_KERNEL_GENERIC = 1, /* two launches per sweep, one per colour; any model */
    LAT_KERNEL_TILED = 2,   /* one launch per sweep, shared-memory tiles with halo
                               recompute; 2D spin-1/2 (Ising and North-East), L % 32 == 0 */
    LAT_KERNEL_WIDE = 3,    /* two launches per sweep, several sites per thread: 2D
                               spin-1/2 (Ising and North-East, L % 32 == 0; with
                               coupling and field signs too), Ising in 3D / with
                               spin S > 1/2 (L % 16 == 0), or Potts (L % 16 == 0) */
    LAT_KERNEL_RESIDENT = 4 /* one launch for many sweeps: one CTA holds the whole
                               lattice in shared memory; 2D spin-1/2 (Ising and
                               North-East), L % 32 == 0, L^2 (+ L^2/4 for North-East)
                               bytes <= 220 KiB, i.e. L <= 448 (Ising) / 416 (NE) */
};

typedef struct lattice lattice_t;
typedef struct lattice_batch lattice_batch_t;
typedef struct lattice_server lattice_server_t;

/* ------------------------------------------------------------------ */
/* Single lattice                                                      */
/* ------------------------------------------------------------------ */

/* Create a lattice on the current CUDA device and write its initial state
 * on the device (§III.A step 1, §III.B step 1 -- done on the GPU here).
 *   dims     2 or 3
 *   L        even, >= 2, L^dims < 2^32
 *   two_S    1..8 (2 * spin); North-East and the bit-packed layout need 1
 *   model    LAT_ISING, LAT_NE (North-East needs dims = 2) or LAT_POTTS
 *            (q = two_S + 1 states; init COLD = all state 0, RANDOM =
 *            uniform labels; for q = 2 the Ising draws, state 0 <-> up)
 *   J, h     coupling and field of H above
 *   T_or_c   temperature (> 0) in energy units, or, for LAT_NE with
 *            J = h = 0, the concentration c in (0, 1)
 *   seed     64-bit Philox key
 *   init     enum lattice_init (EQUILIBRIUM needs LAT_NE with J = h = 0)
 *   layout   enum lattice_layout
 *   cuda_stream  a cudaStream_t, or NULL for the default stream
 * On success *out owns the device memory (spins, persistence bitmap,
 * threshold table, per-sweep counters) until lattice_destroy. */
int lattice_create(lattice_t **out, int dims, int L, int two_S, int model,
                   double J, double h, double T_or_c, uint64_t seed,
                   int init, int layout, void *cuda_stream);

/* Queue n >= 0 checkerboard sweeps (§III.A steps 5-8; §III.B rule) on the
 * handle's stream; returns without waiting.  After each sweep t the four
 * exact int64 counters of lattice_series are recorded on the device. */
int lattice_sweep(lattice_t *lat, int64_t n);

/* Per-site observables of the current configuration (waits for the
 * stream): E/N = (-J*bond - h*mag)/N (mag replaced by the field sum while
 * per-site field signs are set), M/N, up density, and persistence =
 * fraction of sites that never changed since creation or the last
 * lattice_set_state (North-East only; NaN for Ising).  NULL outputs are
 * skipped.  For North-East in c-mode E uses J = 0, h = -1. */
int lattice_observables(lattice_t *lat, double *E, double *M, double *density,
                        double *persistence);

/* Copy the exact per-sweep counters of sweeps [first, first+count) (0-based
 * global sweep index, counted since creation or the last set_state) to the
 * caller's host arrays (NULL arrays are skipped):
 *   bond[k]      sum over sites and directions of s_i * s_{i+e_d}
 *   mag[k]       sum of s_i
 *   up[k]        number of sites with s_i > 0
 *   unflipped[k] number of sites never changed (North-East; 0 for Ising)
 * LAT_ERANGE if the range is not recorded. */
int lattice_series(lattice_t *lat, int64_t first, int64_t count, int64_t *bond,
                   int64_t *mag, int64_t *up, int64_t *unflipped);

/* Spin-spin autocorrelation (§III.B, Eq. 4):
 *   Phi(t) = (1/N) sum_i [s_i(t) s_i(0) - m^2] / (1 - m^2),  m = <s_i> = 2c - 1,
 * with the sum over sites read as the mean, so that Phi(0) = 1 for +-1 spins.
 * lattice_set_reference stores the current configuration as s(0) (a device
 * copy: N bytes, or the bit-packed size) and returns in *ref_sweep (may be
 * NULL) the sweeps done at that moment.  From then on every sweep also
 * records, in the same kernels as the other counters, the exact overlap
 *   overlap = sum_i s_i(t) s_i(0)      (int64)
 * of the state after that sweep.  For the Potts model the overlap is the
 * number of sites whose label equals the reference label, and m = 1/sqrt(q)
 * gives Phi = (overlap/N - 1/q) / (1 - 1/q).  A later call replaces the reference;
 * lattice_clear_reference frees it and stops the recording.  Neither
 * set_state nor set_spins changes the reference. */
int lattice_set_reference(lattice_t *lat, int64_t *ref_sweep);

/* Per-bond couplings (Eq. 1: H = -sum_<ij> J_ij s_i s_j - h sum_i s_i with
 * J_ij = J * eps_ij, eps_ij = +-1: the Edwards-Anderson +-J spin glass).
 * bond_signs holds dims * N int8 values of +-1: bond_signs[d*N + i] is eps
 * for the bond from site i (x fastest) to its +e_d neighbour (periodic).
 * NULL restores uniform couplings.  From then on lattice_series' bond[k] is
 * the weighted sum over bonds of eps_ij s_i s_j, so E = -J*bond - h*mag as
 * before.  Ising model, int8 layout, checkerboard dynamics only
 * (LAT_ENOTSUP otherwise); LAT_EINVAL for values other than +-1.  Such
 * lattices sweep with the 2D wide kernel (2D spin-1/2) or the generic one;
 * the tiled, resident, bit-packed and random-site paths are not available
 * (lattice_set_kernel answers LAT_ENOTSUP).  Uses N bytes of device memory
 * (shared with the field signs below); a checkpoint (lattice_get_state)
 * does not include the couplings.  Waits for the stream. */
int lattice_set_couplings(lattice_t *lat, const int8_t *bond_signs);

/* Per-site random fields (Eq. 1 with B_i = h * eta_i, eta_i = +-1: the
 * random-field Ising model with a bimodal field).  field_signs holds N int8
 * values of +-1, field_signs[i] = eta for site i (x fastest); NULL restores
 * the uniform field.  Couplings and field signs are independent: setting
 * or clearing one keeps the other.  From then on every sweep also records
 *   field = sum_i eta_i s_i       (int64, lattice_field_series)
 * and lattice_observables reports E/N = (-J*bond - h*field)/N.  Same
 * restrictions as lattice_set_couplings; such lattices sweep with the 2D
 * wide kernel (2D spin-1/2, L % 32 == 0) or the generic one, and in a
 * batch with the generic one.  The acceptance table gains a second half
 * for -h.  Waits for the stream; LAT_EINVAL for values other than +-1. */
int lattice_set_fields(lattice_t *lat, const int8_t *field_signs);

/* Copy the recorded field sums of sweeps [first, first+count) to field[]
 * (int64).  LAT_ENOENT when no field signs are set; LAT_ERANGE unless the
 * range was swept with the current field signs and is recorded. */
int lattice_field_series(lattice_t *lat, int64_t first, int64_t count, int64_t *field);

/* Choose the sweep dynamics of later lattice_sweep calls.
 * LAT_DYNAMICS_RANDOM_SITE is the paper's own North-East GPU algorithm
 * (§III.B, steps 3-10, Figs. 4-5), for 2D spin-1/2 int8 lattices of either
 * model: the lattice is cut into tile x tile sub-lattices (tile a power of two
 * in [8, 256] dividing L); one sweep is two launches, and in each launch
 * every sub-lattice makes q rounds of lambda concurrent random picks
 * (lambda a power of two, 1 <= lambda <= min(1024, tile^2/2), q * lambda =
 * tile^2/2), with its boundary frozen at the launch's start.  Randomness:
 * thread i of sub-lattice B (row-major) makes one Philox call per two
 * rounds, rounds 2k and 2k+1 of launch l in sweep t sharing the counter
 * (B*C + k*lambda + i, t lo, t hi, 4 + l) with C = ceil(q/2)*lambda; round r
 * takes word 2(r&1) for the site (floor(w * tile^2 / 2^32), row-major) and
 * word 2(r&1)+1 for the acceptance.  Picks of one round are decided from
 * the state at the round's start; of several picks of one site the lowest
 * thread index's is kept.  tile = L (one sub-lattice) with lambda = 1 is
 * serial random-site Metropolis.
 * LAT_DYNAMICS_RANDOM_SITE_BALANCED is the variant that keeps the weaker
 * balance condition: four launches per sweep (tags 4..7), each making q/2
 * rounds that alternate colour 0 (the paper's red) and colour 1 (white),
 * starting with colour 0; a round's picks are drawn among the tile^2/2
 * sites of its colour (m = floor(w * tile^2/2 / 2^32), row m / (tile/2),
 * column 2 (m mod tile/2) + ((row + colour) & 1)).  It needs q/2 even
 * (lambda <= tile^2/8).  With one sub-lattice it leaves the Boltzmann
 * distribution stationary for any lambda.  Allocates one more lattice-sized buffer (N bytes) the first
 * time.  Counters, persistence and the autocorrelation are recorded as for
 * the checkerboard.  LAT_ENOTSUP for 3D, spin-S or bit-packed lattices,
 * LAT_EINVAL for other tile / lambda values.  Such lattices cannot join a
 * batch (lattice_batch_add: LAT_ENOTSUP). */
int lattice_set_dynamics(lattice_t *lat, int dynamics, int tile, int lambda);
int lattice_clear_reference(lattice_t *lat);
/* Copy the overlaps of sweeps [first, first+count) (global sweep indexes as in
 * lattice_series; first >= the reference's ref_sweep) to overlap[] and, if phi
 * is not NULL, Phi = (overlap/N - m^2) / (1 - m^2) to phi[] (|m| < 1 required,
 * LAT_EINVAL otherwise).  m = NaN asks for the model's own polarisation: for
 * the North-East model at concentration c, m = <s_i> = 2c - 1 (§III.B,
 * Eq. 4); a lattice without one gives LAT_EINVAL when phi is requested.
 * NULL arrays are skipped.  LAT_ENOENT if no reference is set, LAT_ERANGE
 * if the range is not recorded. */
int lattice_autocorrelation(lattice_t *lat, int64_t first, int64_t count, double m,
                            int64_t *overlap, double *phi);

/* Copy the N = L^dims spins (int8, x fastest, spin values) to host_out,
 * whatever the layout (waits for the stream). */
int lattice_get_spins(lattice_t *lat, int8_t *host_out);

/* Replace the spins from a caller host array of N int8 spin values (each
 * must be an allowed value; LAT_EINVAL otherwise).  The persistence flags
 * and the sweep counter are left unchanged. */
int lattice_set_spins(lattice_t *lat, const int8_t *host_in);

/* Checkpoint: spins (N int8), persistence flags (N uint8, 0/1; may be NULL)
 * and the number of sweeps done.  lattice_set_state restores them; the
 * counter-based random numbers make a resumed run bit-exact with an
 * uninterrupted one.  set_state clears the recorded series. */
int lattice_get_state(lattice_t *lat, int8_t *spins, uint8_t *flags, int64_t *sweeps);
int lattice_set_state(lattice_t *lat, const int8_t *spins, const uint8_t *flags,
                      int64_t sweeps);

/* Number of sweeps done, N, and device bytes held by the handle. */
int lattice_info(lattice_t *lat, int64_t *sweeps, int64_t *n_sites, int64_t *device_bytes);

/* Device address and size of the current spin storage, valid until the
 * next sweep (the buffers alternate).  int8 layout: checkerboard-planar,
 * N int8 spins where plane c = (x+y+z) mod 2, row r = y + L*z and
 * j = x >> 1 sit at c*(N/2) + r*(L/2) + j.  Bit-packed layout: 2 colour
 * planes x L rows x ceil(L/64) uint32 words, bit j of a row = site j of
 * that plane row, set = up. */
int lattice_device_spins(lattice_t *lat, void **dev_ptr, size_t *bytes);

/* Pick the kernel (enum lattice_kernel), the tile shape (tile_w columns x
 * tile_h rows; 0 = default) and the sweeps per CUDA-graph replay
 * (0 = default).  LAT_ENOTSUP if the kernel does not cover the lattice.
 * With LAT_KERNEL_AUTO an int8 lattice with uniform couplings is tuned by
 * its first long enough sweep call, on the caller's own sweeps (same bits
 * whichever kernel or graph size runs them):
 *   - the kernel, when there is a choice (2D spin-1/2 with L % 32 == 0:
 *     wide, tiled at two tile heights, resident when it fits one CTA), 8
 *     sweeps per candidate, which needs a call of at least 8 sweeps per
 *     candidate;
 *   - then the sweeps per CUDA-graph replay (a size set here is kept): half,
 *     one, two and four times the default size, each timed on one replay
 *     after an untimed one, as far as the call's remaining sweeps reach.
 * The choice is kept for that (model, dims, two_S, L) for the life of the
 * process.  If the environment variable LATTICE_TUNE_CACHE names a file,
 * the choices also persist there, one JSON object per line:
 * {"model": m, "dims": d, "two_S": s, "L": L, "kernel": k, "tile_h": h,
 *  "graph": g} (g = 0: the default size). */
int lattice_set_kernel(lattice_t *lat, int kernel, int tile_w, int tile_h,
                       int sweeps_per_graph);

/* The kernel actually used for this lattice (enum lattice_kernel, never
 * AUTO), its tile shape (0 when the kernel has none) and the sweeps per
 * CUDA-graph replay.  NULL outputs are skipped. */
int lattice_get_kernel(lattice_t *lat, int *kernel, int *tile_w, int *tile_h,
                       int *sweeps_per_graph);

/* The acceptance table the library builds on the host (no GPU needed) for
 * the given model parameters (same meaning and checks as lattice_create):
 * for ds = s' - s in [-dsmax, dsmax] and neighbour sum n in [-nmax, nmax],
 * entry (ds + dsmax) * (2 nmax + 1) + (n + nmax) holds always (1 = accept
 * without a draw) and thr (accept iff u < thr).  Writes at most cap
 * entries (thr / always may be NULL); *count, *dsmax, *nmax receive the
 * table size and ranges. */
int lattice_threshold_table(int dims, int two_S, int model, double J, double h, double T_or_c,
                            uint32_t *thr, uint8_t *always, int cap, int *count, int *dsmax,
                            int *nmax);

/* Wait for all queued work of the handle. */
int lattice_synchronize(lattice_t *lat);

void lattice_destroy(lattice_t *lat);

/* ------------------------------------------------------------------ */
/* Batch: many lattices (any sizes and models) advanced by one          */
/* persistent-kernel launch per sweep step, replayed from a CUDA graph. */
/* Results are bit-exact with running each lattice alone.               */
/* ------------------------------------------------------------------ */

/* A batch runs on its own stream (NULL = default stream).  Work already
 * queued on a lattice's own stream is ordered before the batch's (an event
 * wait: the host does not block). */
int lattice_batch_create(lattice_batch_t **out, void *cuda_stream);
/* Schedule n more sweeps of lat in the next lattice_batch_run. */
int lattice_batch_add(lattice_batch_t *b, lattice_t *lat, int64_t n);
/* Run every scheduled sweep; returns after queueing (lattice_synchronize
 * or lattice_batch_synchronize waits: each lattice's stream is made to wait
 * for the batch).  Lattices with fewer remaining sweeps drop out of later
 * launches.  2D spin-1/2 lattices with L <= 128 (under LAT_KERNEL_AUTO) or
 * set to LAT_KERNEL_RESIDENT run as resident CTAs, one per lattice, for all
 * their sweeps, concurrently with the others. */
int lattice_batch_run(lattice_batch_t *b);
int lattice_batch_synchronize(lattice_batch_t *b);
/* The batch engine's two tunables as its last run used them: the rows a
 * thread visits per item of the pipelined 2D spin-1/2 kernel
 * (*rows_per_item; 0 = the size-based default, 8 rows on lattices with
 * L >= 1024 and 2 below; the 3D / spin-S and Potts items size themselves
 * to the phase's work of their kind, 4 to 32 rows) and the steps per
 * captured CUDA graph (*steps_per_graph).  A run whose first phase (all its
 * lattices) has at least 192 steps tunes both once per composition of
 * lattices (models, dimensions, spins, sizes and kernels), timing
 * candidates on its own steps (same bits whichever runs) and synchronising
 * the host meanwhile; shorter runs use the tuned values of their
 * composition, or the defaults.  NULL outputs are skipped. */
int lattice_batch_tuning(lattice_batch_t *b, int *rows_per_item, int *steps_per_graph);
void lattice_batch_destroy(lattice_batch_t *b);

/* ------------------------------------------------------------------ */
/* Server: continuous batching of independent simulation requests.     */
/* ------------------------------------------------------------------ */
typedef struct lattice_request {
    int dims, L, two_S, model;      /* as lattice_create */
    double J, h, T_or_c;
    uint64_t seed;
    int init;
    int64_t sweeps;                 /* sweeps to run, >= 0 */
    int keep_spins;                 /* 1: keep the final spins for lattice_server_poll */
} lattice_request_t;

typedef struct lattice_result {
    int status;             /* LAT_OK, or the error that ended the request */
    int64_t sweeps_done;
    int64_t bond, mag, up, unflipped;  /* counters after the last sweep */
    double E, M, density, persistence; /* per site, as lattice_observables */
    double t_submit, t_admit, t_done;  /* seconds on the server's clock */
} lattice_result_t;

/* A server owns two CUDA streams (on the device current at creation: one
 * for the batched rounds, one for creating, reading back and freeing
 * lattices) and one scheduler thread.  Requests wait in arrival order and
 * are admitted while their device footprint fits in hbm_budget_bytes and
 * fewer than max_slots lattices are resident.  Each scheduling round
 * advances every resident lattice by up to chunk_sweeps sweeps through the
 * batched engine (so work of requests that arrived at different times
 * shares launches).  Rounds are pipelined: the next round is queued while
 * the current one runs, and admission, lattice creation and the retirement
 * of finished lattices (read-back, freeing their memory) happen meanwhile.
 * Every result is bit-identical to running its lattice alone.  This is
 * continuous batching: admission happens between rounds, never by stopping
 * resident work.  A request whose lattice cannot be created or queued
 * (e.g. LAT_ENOMEM) ends with that status alone; a failed launch ends the
 * requests of its round with LAT_ECUDA. */
int lattice_server_create(lattice_server_t **out, size_t hbm_budget_bytes, int max_slots,
                          int chunk_sweeps);
/* Non-blocking; *id identifies the request. LAT_EINVAL for a bad request,
 * LAT_ENOMEM if it can never fit the budget. */
int lattice_server_submit(lattice_server_t *s, const lattice_request_t *req, uint64_t *id);
/* LAT_EBUSY until done; then fills *res and, if spins_out is not NULL,
 * copies the final N spins there.  A finished result can be polled once
 * more after which it is released (LAT_ENOENT). */
int lattice_server_poll(lattice_server_t *s, uint64_t id, lattice_result_t *res,
                        int8_t *spins_out);
/* Block until every submitted request is finished (or timeout_s seconds,
 * LAT_ETIMEOUT; timeout_s <= 0 waits without limit). */
int lattice_server_drain(lattice_server_t *s, double timeout_s);
/* Seconds on the server's clock (same clock as lattice_result times). */
double lattice_server_clock(lattice_server_t *s);
/* Device time of the rounds run so far (*busy_s, from CUDA events around
 * each round's device work), the server's clock (*wall_s) and the number of
 * rounds; busy / wall is the fraction of time the GPU worked for the server.
 * NULL outputs are skipped. */
int lattice_server_stats(lattice_server_t *s, double *busy_s, double *wall_s, int64_t *rounds);
void lattice_server_destroy(lattice_server_t *s);

/* ------------------------------------------------------------------ */
/* No-allocation batched sweep (this entry point has no counterpart in  */
/* the paper; it serves callers that cannot let a library allocate).    */
/* ------------------------------------------------------------------ */

/* One 2D spin-1/2 Ising lattice (H = -J sum s_i s_j - h sum s_i, same
 * rules, random numbers and counters as lattice_create / lattice_sweep)
 * held entirely in caller-owned device memory:
 *   L         lattice side, a multiple of 32, 32 <= L <= 32768
 *   J, h, T   coupling, field, temperature (T > 0; the acceptance table
 *             must not contain a never-accept entry, i.e. dE/T <= 22)
 *   seed      Philox key
 *   sweep0    sweeps already done (global sweep index of the first sweep)
 *   spins[2]  two device buffers of L*L int8 spins each, in the
 *             checkerboard-planar layout of lattice_device_spins; the state
 *             after t sweeps is in spins[t & 1] (the other is overwritten)
 *   counters  device int64[4 * n_sweeps]: bond, mag, up, unflipped (0) of
 *             each sweep, in order; cleared by the call before use */
typedef struct lattice_static_desc {
    int L;
    double J, h, T;
    uint64_t seed;
    int64_t sweep0;
    int8_t *spins[2];
    int64_t *counters;
} lattice_static_desc_t;

/* Queue n_sweeps checkerboard sweeps of n_lattices lattices on cuda_stream
 * (NULL = default stream) without allocating any memory: no cudaMalloc,
 * cudaFree or allocating library call.  For callers whose device memory
 * all comes from their own pool (a framework's caching allocator, a
 * memory-capped service) or that must not trigger the device-wide
 * synchronisation an allocation can cause.
 *   - The library's scratch (descriptors, tables, sweep counters, the tile
 *     work list) is one fixed array of about 560 kB in device memory that
 *     every GPU loading the library holds until the process exits.  Limits:
 *     at most 64 lattices and 65536 tiles of 256 x 64 sites per call
 *     (LAT_ERANGE beyond either; one L = 32768 lattice is 65536 tiles).
 *   - The first call on a device looks up the scratch's address (with that
 *     device current); make that first call before any stream capture.
 *   - All calls share the scratch, which keeps the last call's contents;
 *     the call clears what must start at zero.  Calls whose work overlaps
 *     on the GPU (for example on two streams, or from two host threads)
 *     race on the scratch: serialise them.
 *   - The descriptors are copied from host memory on cuda_stream, and the
 *     call then synchronises cuda_stream before it queues the sweeps: it
 *     blocks until all work queued earlier on that stream (the previous
 *     call's sweeps included) has finished.  It returns without waiting
 *     for the sweeps it queues.
 * Returns LAT_EINVAL / LAT_ENOTSUP for bad or unsupported lattices. */
int lattice_sweep_static(const lattice_static_desc_t *descs, int n_lattices, int64_t n_sweeps,
                         void *cuda_stream);

/* ------------------------------------------------------------------ */
const char *lattice_strerror(int code);
/* The last CUDA error string seen by the calling thread (or ""). */
const char *lattice_last_cuda_error(void);
/* Library version string. */
const char *lattice_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LATTICE_H */
