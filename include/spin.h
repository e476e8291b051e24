/*
 * spin.h -- C ABI of the GB300 checkerboard Metropolis library.
 *
 * The library implements the data-parallel hot path of M. Weigel,
 * "Performance potential for simulating spin models on GPU"
 * (arXiv:1101.1427): checkerboard (red-black) Metropolis sweeps for the
 * 2D/3D Ising ferromagnet (Eq. ising_hamiltonian, Eq. metropolis, Sec. 3.2),
 * the +-J Edwards-Anderson spin glass (Eq. spinglass_hamiltonian, Sec. 5,
 * including asynchronous multi-spin coding), the 3D Heisenberg model
 * (Eq. On_hamiltonian, Sec. 4) and the replica-exchange step of parallel
 * tempering (Eq. parallel_tempering, Sec. 6), plus the energy,
 * magnetisation and overlap reductions.
 *
 * Conventions (shared with the test oracle, which implements them
 * independently):
 *   - a lattice has L^dim sites, x fastest, periodic boundaries, L even;
 *     site i = (z*L + y)*L + x; colour c = (x + y + z) mod 2; colour 0 is
 *     swept first; j = i >> 1 indexes a site inside its colour.
 *   - random words come from Philox4x32-10 with key (seed lo, seed hi) and
 *     counter (idx >> 2, sweep, lattice_id, tag << 28 | colour << 27 | extra);
 *     word idx & 3 is used.  lattice_id = a << 24 | rkey << 12 | t for
 *     replica set a, temperature slot t and realisation key rkey (the
 *     realisation r for Ising/Heisenberg lattices, the group r >> 5 for EA).
 *   - Ising/EA acceptance: flip iff dE <= 0 or r < thr(dE), with the integer
 *     threshold thr(dE) = min(2^32 - 1, floor(exp(-beta dE) 2^32)) computed
 *     on the host in double precision.  Ising and EA trajectories are
 *     therefore exact integer functions of (seed, inputs).
 *
 * Ownership: every spin, coupling and output buffer is allocated and owned
 * by the caller; the library only borrows device pointers while the work it
 * enqueued on the handle's stream runs.  A handle owns small workspaces
 * (threshold tables, reduction partials, an error word), allocated by
 * spin_init, and one lattice-sized working buffer allocated by the first
 * sweep call that needs it (the fused 2D int8 pass, the coded path of int8
 * lattices, long Heisenberg calls), with, for the resident 3D Heisenberg
 * sweeps, one counter per CTA; all are freed by spin_destroy.
 *
 * Errors: every entry point returns 0 (SPIN_OK) or a negative SPIN_E* code
 * and never throws.  Work is asynchronous on the handle's stream; kernel
 * faults and device-side timeouts surface from spin_sync (or the next call).
 */
#ifndef SPIN_GB300_H
#define SPIN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPIN_OK 0
#define SPIN_EINVAL (-1)   /* bad argument: odd L, bad layout/model, NaN beta ... */
#define SPIN_EALIGN (-2)   /* a device pointer is not 16-byte aligned            */
#define SPIN_ENOMEM (-3)   /* workspace allocation failed                        */
#define SPIN_ECUDA (-4)    /* a CUDA runtime call or kernel failed               */
#define SPIN_ETIMEOUT (-5) /* a bounded device-side wait gave up                 */

typedef enum { SPIN_ISING = 0, SPIN_EA = 1, SPIN_HEISENBERG = 2 } spin_model;

/* Storage of the spins in device memory (lat = (a * n_temps + t) * n_real + r):
 *  SPIN_I8     int8 +-1, [n_sets][n_temps][n_real][L^dim].  Ising (2D, 3D) and
 *              EA (3D, one spin per byte: the per-realisation form).
 *  SPIN_MSC1   1 bit per spin, bit set <=> s = -1, uint32 words.
 *              EA (2D or 3D, asynchronous coding, Sec. 5): word-lattices
 *              [n_sets][n_real/32][n_temps], each stored colour-split as
 *              [2 colours][L^dim/2] (site i of colour c at c L^dim/2 + (i >> 1));
 *              bit b of a word is realisation 32 g + b.
 *              Ising 2D ferromagnet (synchronous coding): per lattice
 *              [2 colours][L rows][L/64 words]; in row y the colour-c sites
 *              x = 2k + ((c + y) & 1) are grouped in blocks of 128 k's, and
 *              k = 128 B + 4 l + q is bit l of word 4 B + q.  Needs L % 256 == 0.
 *  SPIN_F32X4  float4 (x, y, z, 0) unit vectors, [n_sets][n_temps][n_real][L^dim]
 *              (Heisenberg, 2D as in Sec. 4 or 3D).
 * Couplings (EA only; NULL for the ferromagnet, J = 1):
 *  SPIN_I8     int8 +-1, [n_real][dim][L^dim]: bond (i, i + e_d).
 *  SPIN_MSC1   uint32 [n_real/32][dim][2 colours][L^dim/2] (bond (i, i + e_d)
 *              at d L^dim + c(i) L^dim/2 + (i >> 1)), bit b set <=> J = -1 for
 *              realisation 32 g + b.
 * All device buffers must be 16-byte aligned. */
typedef enum { SPIN_I8 = 0, SPIN_MSC1 = 1, SPIN_F32X4 = 2 } spin_layout;

typedef struct {
  int32_t model;     /* spin_model                                             */
  int32_t dim;       /* 2 or 3                                                 */
  int32_t L;         /* edge length: even, >= 4                                */
  int32_t layout;    /* spin_layout                                            */
  int32_t n_real;    /* lattices per (set, slot): EA disorder realisations     */
                     /* (multiple of 32 for MSC1) or independent lattices      */
  int32_t n_temps;   /* temperature slots (>= 1, <= 4096)                      */
  int32_t n_sets;    /* replica sets (>= 1, <= 255; 2 for the overlap)         */
  int32_t hot_start; /* 1: random start from the seed; 0: all spins +1 (+z)    */
  uint64_t seed;     /* Philox key for every random number of this handle      */
  void *stream;      /* cudaStream_t for all work of this handle; NULL = default */
} spin_desc;

typedef struct spin_lattice spin_lattice; /* opaque handle */

/* Creates a handle for the caller-owned device buffers `spins` and
 * `couplings` (NULL for the ferromagnet and Heisenberg) and enqueues their
 * initialisation: spins from the INIT stream (hot start) or all +1, EA
 * couplings from the COUPLING stream (bimodal, Eq. spinglass_hamiltonian).
 * The sweep and exchange counters start at 0. */
int spin_init(spin_lattice **out, const spin_desc *desc, void *spins, void *couplings);

/* n_sweeps checkerboard sweeps (Sec. 3.2; all colour-0 sites, then all
 * colour-1 sites, each with Eq. metropolis or, for the Heisenberg model, a
 * uniformly drawn new direction accepted with Eq. metropolis).  betas is a
 * HOST array of n_temps inverse temperatures (beta >= 0, finite); couplings
 * as in spin_init.  seed must equal the handle's seed (else SPIN_EINVAL).
 * Sweep k of this call uses sweep counter value (sweeps done so far) + k, so
 * consecutive calls continue one Markov chain.  Heisenberg spins are
 * renormalised after every sweep whose 1-based count is a multiple of 100.
 * The per-handle calls take their sweep numbers from the host counter when
 * they are enqueued, so a CUDA graph captured around them would repeat the
 * same random numbers on every replay; the batched launch (spin_batch_run)
 * reads its counters on the device and is the form meant for capture. */
int spin_sweep(spin_lattice *lat, const void *couplings, const double *betas,
               int64_t n_sweeps, uint64_t seed);

/* Reductions over the current state (Sec. 3.5, measurement by binary-tree
 * reduction; double accumulation for continuous spins, Sec. 4).  Device
 * outputs, NULL to skip; lat index = (a * n_temps + t) * n_real + r:
 *   E   int64 [n_lat]  E = -sum_<ij> J_ij s_i s_j        (Ising, EA)
 *   M   int64 [n_lat]  M = sum_i s_i                     (Ising, EA)
 *   Q   int64 [n_temps][n_real]  q = sum_i s_i^(0) s_i^(1) between sets 0, 1 (EA)
 *   Ef  double [n_lat]     E = -sum_<ij> s_i . s_j       (Heisenberg)
 *   Mf  double [n_lat][3]  M = sum_i s_i                 (Heisenberg) */
int spin_measure(spin_lattice *lat, const void *couplings, int64_t *E, int64_t *M,
                 int64_t *Q, double *Ef, double *Mf);

/* One replica-exchange step (Eq. parallel_tempering) for Ising/EA handles:
 * for every set a and realisation r, the slot pairs (t, t+1) with
 * t = p (mod 2), p the handle's exchange counter, are tried with
 * Delta = (beta_{t+1} - beta_t)(E_{t+1} - E_t): accepted iff Delta >= 0 or
 * the PT word r < floor(exp(Delta) 2^32).  Accepted pairs exchange their
 * configurations (bitwise for MSC1).  Energies are computed on the device
 * from the current state.  accepted (device int64 [n_sets][n_temps], may be
 * NULL) is incremented per accepted pair (t, t+1) at index t.  labels
 * (device int32 [n_sets][n_temps][n_real], indexed like the lattices, may be
 * NULL) names the configuration each lattice holds: an accepted exchange
 * moves the two labels with their configurations.  Sec. 6 notes that
 * exchanging temperatures instead of configurations is cheaper on a CPU;
 * the labels give a caller of this configuration-exchange form the same
 * information -- starting from labels[lat(a, t, r)] = t, the slot of every
 * configuration (slot_of_config, for round-trip counts) is the inverse
 * permutation of labels over t for each (a, r).  The values are the
 * caller's; the library only moves them.  The exchange counter then
 * advances by one. */
int spin_pt_swap(spin_lattice *lat, const void *couplings, const double *betas,
                 uint64_t seed, int64_t *accepted, int32_t *labels);

/* A whole simulation on one handle: n_sweeps sweeps; after every sweep that
 * brings the handle's sweep count (spin_sweeps_done) to a multiple of
 * measure_every (> 0) the measurements of spin_measure are appended to the
 * series (device buffers, NULL to skip, row k holds the call's measurement
 * k, so a call writes (s + n_sweeps) / measure_every - s / measure_every
 * rows for a count s before it); after every sweep that brings the count to
 * a multiple of pt_every (> 0) one exchange step as in spin_pt_swap follows
 * the measurement; accepted and labels as in spin_pt_swap. */
int spin_run(spin_lattice *lat, const void *couplings, const double *betas, int64_t n_sweeps,
             int32_t measure_every, int32_t pt_every, int64_t *E_series, int64_t *M_series,
             int64_t *Q_series, double *Ef_series, double *Mf_series, int64_t *accepted,
             int32_t *labels);

/* One handle of a batched launch: its couplings and HOST betas as in
 * spin_sweep, and optional device series, counters and configuration
 * labels as in spin_run. */
typedef struct {
  spin_lattice *lat;
  const void *couplings;
  const double *betas;
  int64_t *E_series;
  int64_t *M_series;
  int64_t *Q_series;
  int64_t *accepted;
  int32_t *labels;
} spin_batch_item;

/* Batched persistent launch (the paper maps independent replicas and
 * tempering copies to thread blocks, Sec. 5-6): n_sweeps sweeps of every
 * lattice of every handle, with the measurements and exchange steps of
 * spin_run, in ONE cooperative kernel launch on `stream`.  Results
 * (lattices, series, exchange decisions) are identical to calling spin_run
 * on each handle.  Supported handles: 3D EA in the coded layout (L <= 32) and
 * 2D ferromagnets, int8 with L % 16 == 0 or coded with L % 256 == 0, in the
 * checkerboard order and without exchange between their slots; at most 16
 * handles and 96 work units (one unit per EA realisation group or Ising
 * lattice).  Work units are spread over teams of co-resident CTAs in
 * proportion to their work; a team synchronises through global-memory
 * barriers whose waits are bounded in time: on expiry the launch ends early
 * and spin_sync on the FIRST item's handle returns SPIN_ETIMEOUT.
 *
 * The launch reads each handle's sweep and exchange counters from a device
 * copy and advances that copy when it ends (both in stream order), so the
 * work one call enqueues can be captured into a CUDA graph and replayed:
 * each replay continues the random streams where the previous one ended.
 * An uncaptured call uploads the tables for `betas` if they changed,
 * allocates the handle's batch workspace on first use (kept until
 * spin_destroy) and loads the device counters from the host counters;
 * n_sweeps = 0 does only that.  Inside a stream capture the call uploads and
 * allocates nothing and returns SPIN_EINVAL unless an uncaptured call with
 * the same betas came first, no other call has moved the counters since,
 * and measure_every (if > 0) divides n_sweeps.  Capturing advances the host
 * counters once, as if the captured work had run; a caller that replays the
 * graph R times sets them (spin_set_counters) to the values after R runs.
 * Changing a handle's betas after the capture invalidates the graph. */
int spin_batch_run(const spin_batch_item *items, int n_items, int64_t n_sweeps,
                   int32_t measure_every, int32_t pt_every, void *stream);

/* Autotuner for spin_batch_run: times n_sweeps-sweep trial launches (with
 * the given measurement and exchange schedule, into scratch series) for
 * 1..4 CTAs per SM and the weights of the split of CTAs between work units
 * (three weights of the Ising units when the batch mixes Ising and EA
 * handles; three fixed costs per EA word-lattice, 0, 1024 and 4096 sites,
 * when its EA lattices have several sizes), on copies of the spins (handles
 * and counters are left as they were), and caches the fastest choice for
 * this batch shape; best (optional, host) receives the CTAs per SM.  The
 * choice changes only which CTAs do which work, never the results. */
int spin_batch_tune(const spin_batch_item *items, int n_items, int64_t n_sweeps,
                    int32_t measure_every, int32_t pt_every, void *stream, int32_t *best);

/* Batch options taken from the first item's handle: bound on every barrier
 * wait in ns (0: 2 s), CTAs per SM (0: autotuned or 2), and a number of
 * barrier arrivals that never come (0 in normal use; > 0 makes every team
 * barrier wait out its bound, for tests of the timeout path).  The bound
 * and the missing arrivals also apply to the neighbour waits of the resident
 * 3D Heisenberg sweeps (spin_set_variant); a wait that runs out ends the
 * launch early (the lattices keep their contents from before the call) and
 * spin_sync reports SPIN_ETIMEOUT. */
int spin_set_batch_options(spin_lattice *lat, uint64_t timeout_ns, int32_t ctas_per_sm,
                           int32_t missing_arrivals);

/* Layout conversion between the handle's layout and one int8 spin per site
 * ([n_sets][n_temps][n_real][L^dim], +-1), device buffers. */
int spin_unpack_i8(spin_lattice *lat, int8_t *out);
int spin_pack_i8(spin_lattice *lat, const int8_t *in);

/* Counter-based random words, exactly as the kernels draw them:
 * out[k] = word k & 3 of Philox4x32-10(counter (k >> 2, sweep, lattice_id,
 * tag << 28 | colour << 27 | extra), key (seed lo, seed hi)), k < count.
 * out is a device buffer; the work runs on `stream`. */
int spin_rng_fill(uint64_t seed, uint32_t tag, uint32_t colour, uint32_t extra,
                  uint32_t lattice_id, uint32_t sweep, uint64_t count, uint32_t *out,
                  void *stream);

/* Generator throughput probe (the paper times its generators alone, Sec. 3.3):
 * thread k < threads evaluates `calls` Philox4x32-10 blocks with counters
 * (k + i * threads, 0, 0, 0), i < calls, key (seed lo, seed hi), and writes
 * the XOR of all their words to out[k] (device buffer of `threads` words).
 * threads * calls must stay below 2^32. */
int spin_rng_probe(uint64_t seed, uint32_t threads, uint32_t calls, uint32_t *out, void *stream);

/* Instruction-throughput probe for the roofline of the sweeps (the
 * operations of Philox4x32-10 and of the updates; no counterpart in the
 * paper).  Launches blocks_per_sm CTAs of 256 threads on every SM; every
 * thread g (global index) keeps eight chains x[c], c < 8, and runs `iters`
 * iterations of one operation on all eight:
 *   SPIN_PIPE_MUL_WIDE  64-bit x[c] = lo32(x[c]) * 0xD2511F53 + x[c] (mad.wide.u32), x[c] = 8 g + c + 1
 *   SPIN_PIPE_MAD_HI    x[c] = hi32(x[c] * 0xCD9E8D57) + 0x9E3779B9 (mad.hi.u32), x[c] = 8 g + c + 1
 *   SPIN_PIPE_LOP3      x'[c] = x[c] ^ x[c+1] ^ x[c+2] (indices mod 8, all from the old x; lop3.b32), x[c] = 8 g + c + 1
 *   SPIN_PIPE_IADD3     x'[c] = x[c] + x[c+1] + x[c+2] mod 2^32 (as LOP3), x[c] = 8 g + c + 1
 *   SPIN_PIPE_FFMA      x[c] = fma(x[c], 0.999f, 0.001f), x[c] = 1 + (8 g + c) 2^-20 (FP32)
 *   SPIN_PIPE_MUFU_RSQ  x[c] = rsqrt.approx.ftz(x[c]), same start (FP32)
 * (8 operations per iteration), then writes sink[g] = XOR over c of x[c]
 * (MUL_WIDE: of lo32 ^ hi32; FFMA, MUFU_RSQ: the bits of the FP32 sum
 * x[0] + ... + x[7], added in that order), and for every CTA b
 * clocks[3b] and clocks[3b + 1], the SM clock (clock64) after the barriers
 * before and after the loop, and clocks[3b + 2], the index of its SM.  The
 * CTAs of one SM do not progress evenly, so the rate of SM m is
 * 256 * 8 * iters * (its CTAs) / (latest end - earliest start over its CTAs)
 * operations per clock.  clocks (int64, 3 per CTA, SMs * blocks_per_sm CTAs)
 * and sink (uint32, 256 entries per CTA) are caller-owned device buffers;
 * `sms` returns the SM count (host pointer, may be NULL).  SPIN_EINVAL if op
 * is unknown, blocks_per_sm is outside 1..8 or that many CTAs of this kernel
 * cannot be resident on one SM together. */
typedef enum {
  SPIN_PIPE_MUL_WIDE = 0,
  SPIN_PIPE_MAD_HI = 1,
  SPIN_PIPE_LOP3 = 2,
  SPIN_PIPE_IADD3 = 3,
  SPIN_PIPE_FFMA = 4,
  SPIN_PIPE_MUFU_RSQ = 5
} spin_pipe_op;
int spin_pipe_probe(int op, int32_t blocks_per_sm, uint32_t iters, int64_t *clocks, uint32_t *sink,
                    int32_t *sms, void *stream);

/* Heisenberg energy and magnetisation (as Ef and Mf of spin_measure, with
 * the same arithmetic and summation order, so the results are bit-identical)
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart; this entry point exists for library users: code inside a
 * framework that owns the whole device-memory pool (a raw cudaMalloc there
 * fails or fragments the pool) and code that must not stall the device
 * (cudaFree, and often cudaMalloc, synchronise it).  It needs no handle:
 * spins is a device float4 array [n_lat][L^dim] (16-byte aligned) on the
 * square (dim = 2) or simple cubic (dim = 3) lattice, Ef [n_lat] and
 * Mf [n_lat][3] are caller-owned device outputs (NULL to skip); work runs on
 * `stream`.  Partial sums live in one fixed array compiled into the library:
 * 256 lattices x 64 blocks x 4 doubles = 512 KiB on every GPU that loads the
 * library, held until process exit.  SPIN_EINVAL for dim other than 2 or 3,
 * odd L or L < 4, n_lat > 256, L^dim >= 2^31 or n_lat L^dim >= 2^31;
 * nothing is allocated, neither by this call nor by any library routine it
 * uses.  The first call on a device looks up the array's device address
 * (one-time set-up per device); make that first call before any stream
 * capture.  Every call overwrites the partial sums before reading them, so
 * no state has to be cleared between calls, but all calls share the one
 * array: calls whose work overlaps on the GPU (different streams without
 * ordering) race and give wrong sums. */
int spin_heis_measure_noalloc(const float *spins, int32_t dim, int32_t L, int32_t n_lat, double *Ef,
                              double *Mf, void *stream);

/* Waits for the handle's stream and reports asynchronous failures
 * (SPIN_ECUDA, SPIN_ETIMEOUT).  Clears the device error word. */
int spin_sync(spin_lattice *lat);

/* Counters and tuning of a handle.  spin_set_counters sets the host
 * counters and, once the handle has a batch workspace, also enqueues on the
 * handle's stream a write of the same values to the device copy that
 * batched launches read. */
int64_t spin_sweeps_done(const spin_lattice *lat);
/* Copies the handle's descriptor (as given to spin_init) to *out (host), so
 * that a binding can size and check the arrays it passes: betas holds
 * n_temps doubles, E and M n_lat int64 per measurement, and so on.
 * SPIN_EINVAL for a NULL argument. */
int spin_describe(const spin_lattice *lat, spin_desc *out);
int64_t spin_pt_steps_done(const spin_lattice *lat);
int spin_set_counters(spin_lattice *lat, int64_t sweeps_done, int64_t pt_steps_done);

/* Kernel variant.  2D int8 ferromagnet: 0 = two in-place colour phases per
 * sweep, 1 = one fused out-of-place pass per sweep (default for L > 128
 * with L % 256 != 0), 3 = resident: one CTA per lattice holds the whole
 * lattice in shared memory for all sweeps of a call and measures E and M
 * itself (default for L % 8 == 0, L <= 128; the paper's tempering code
 * likewise maps replicas to thread blocks, Sec. 6), 4 = coded: a call of at
 * least 4 sweeps packs the lattices into a handle-owned 1-bit buffer
 * (L^2 / 8 bytes per lattice, allocated on first use, kept until
 * spin_destroy), runs the synchronous multi-spin-coded sweep (Sec. 5) and
 * unpacks them, shorter calls take the fused pass (default for
 * L % 256 == 0, L > 128); all four give identical results.  3D int8
 * ferromagnet: 0 = colour phases, 3 = resident (default for L % 8 == 0,
 * L <= 24), identical results.  Heisenberg: 0 = the full-accuracy FP32
 * library functions (default), 2 = the paper's "fast_math" mode (Sec. 4):
 * rho = sqrt(1 - z^2) from the hardware reciprocal square root, sin and cos
 * of the azimuth from the hardware sine and cosine on [-pi, pi), and the
 * acceptance as u3 2^24 < 2^(24 - beta log2(e) dE) with the hardware exp2;
 * within the same tolerances of the FP64 reference.  Calls of at least 4
 * sweeps in variant 2 run on a colour-split copy of the lattices (same
 * results bit for bit).  In either variant, calls of at least 4 sweeps of 3D
 * lattices with L = 64 or 128 that fit in the SMs' shared memory (one
 * lattice of L = 128 on a GPU with at least 145 SMs of 227 KB; up to a few
 * of L = 64) run resident: one cooperative launch per 100-sweep
 * renormalisation interval, each CTA holding a pencil of rows of one lattice
 * in shared memory for all its sweeps and exchanging the pencil's faces with
 * its four neighbours through the handle's lattice-sized working buffer
 * (same results bit for bit; if the GPU refuses the cooperative launch, its
 * SMs shared with other work, the handle takes the other paths from then
 * on).  Inside a stream capture Heisenberg sweeps always take the per-phase
 * kernels (same results; nothing allocated). */
int spin_set_variant(spin_lattice *lat, int32_t variant);

/* Slab decomposition of one 2D int8 ferromagnet over several GPUs (the
 * domain decomposition of Sec. 3.2 carried one level up, to devices): a rank
 * owns rows y0 .. y0 + rows - 1 of the L x L periodic lattice (0 <= y0,
 * y0 + rows <= L) and holds them as a device buffer slab[rows + 2][L] of +-1
 * bytes (8-byte aligned), slab rows 0 and rows + 1 being copies of global
 * rows y0 - 1 and y0 + rows (mod L).  The caller refreshes those two ghost
 * rows from the neighbouring ranks before every colour phase (one row per
 * neighbour; see paper_1101_1427_gb300/slab.py).
 *
 * spin_slab_phase: one colour phase (colour 0 or 1) of the own rows, as in
 * spin_sweep: the colour of a site is that of its global index and its
 * uniform is the UPDATE word of (seed, lattice_id, sweep, global colour
 * index), so the slabs of a lattice together reproduce the unsplit sweep bit
 * for bit.  L % 8 == 0; beta >= 0; work is enqueued on `stream`; ghost rows
 * are read only.
 * spin_slab_measure: device int64 partial sums of the own rows, E over the
 * bond to the right and the bond below of every own site (the last own row
 * reads the lower ghost), M over own sites; the partials of all slabs add up
 * to the lattice's E and M.  Errors: SPIN_EINVAL for bad sizes or pointers,
 * SPIN_EALIGN for a misaligned slab, SPIN_ECUDA for a launch failure.
 * The paper has no multi-GPU code; this is the design its tiling implies. */
int spin_slab_phase(int8_t *slab, int32_t L, int32_t y0, int32_t rows, double beta, uint64_t seed,
                    uint32_t lattice_id, uint32_t sweep, int32_t colour, void *stream);
int spin_slab_measure(const int8_t *slab, int32_t L, int32_t rows, int64_t *E, int64_t *M, void *stream);

/* Realisations that share one uniform per site in the coded EA layout
 * (Sec. 5, footnote: the same random number serves all w spins of a word):
 * 32 (one word, the default) or 64 (the paper's w = 64: realisation groups
 * 2q and 2q + 1 draw the words of group q, i.e. lattice_id(a, r >> 6, t);
 * the storage stays 32-bit, since on this GPU a 64-bit logical operation is
 * two 32-bit ones, and one Philox call serves both words).  Needs n_real a
 * multiple of 64; initial states, couplings and exchange draws do not
 * change. */
int spin_set_msc_width(spin_lattice *lat, int32_t width);

/* Update order of the sweeps of a handle.
 *  SPIN_ORDER_CHECKERBOARD  all colour-0 sites, then all colour-1 sites
 *                           (default; every other call here assumes it).
 *  SPIN_ORDER_DCB           double checkerboard with multi-hit updates
 *                           (Sec. 3.2, Fig. checker; Sec. 3.4): the lattice
 *                           is cut into tile x tile tiles coloured like a
 *                           checkerboard; a compound move gives the tiles of
 *                           coarse colour 0 `hits` hits (fine colour 0,
 *                           then fine colour 1, each hit) and then the
 *                           tiles of coarse colour 1 the same way, so every
 *                           site takes `hits` updates.  Hit h of compound
 *                           move m draws with sweep number m * hits + h.
 *  SPIN_ORDER_DCB_SYMMETRIC the same with coarse colour 1 first in odd
 *                           compound moves (counted by sweeps / hits), so
 *                           that the moves alternate A^k B^k and B^k A^k,
 *                           the compound order of Sec. 3.4 that satisfies
 *                           detailed balance.
 * The double-checkerboard orders take Ising ferromagnets in the int8
 * layout: 2D with tile in {8, 16, 32, 64, 128}, or 3D (Sec. 3.6: tile^3
 * cubes, coarse colour (x / tile + y / tile + z / tile) mod 2) with tile in
 * {8, 16}; and the 2D Heisenberg model (Sec. 4) with tile in {8, 16, 32},
 * renormalised after every compound move that passes a sweep count
 * divisible by 100; tile divides L with L / tile even, and hits >= 1; spin_sweep then counts sweeps as updates per site and needs
 * n_sweeps and the handle's sweep count to be multiples of hits (so must
 * spin_run's measure_every and pt_every).  Such handles cannot join a
 * batched launch.  tile and hits are ignored for SPIN_ORDER_CHECKERBOARD. */
/* tile 0 leaves the tile edge to spin_tune, which must then run before the
 * first sweep (a sweep with the edge still open returns SPIN_EINVAL). */
typedef enum {
  SPIN_ORDER_CHECKERBOARD = 0,
  SPIN_ORDER_DCB = 1,
  SPIN_ORDER_DCB_SYMMETRIC = 2
} spin_update_order;
int spin_set_update_order(spin_lattice *lat, int32_t order, int32_t tile, int32_t hits);

/* Autotuner for one handle (no counterpart in the paper's code; Sec. 3.5
 * chooses its tile size by measuring): times trial calls of n_sweeps sweeps
 * (1 .. 100000; a multiple of the hits in the double-checkerboard order)
 * with the given couplings and HOST betas for every choice that leaves the
 * handle's chain unchanged -- the kernel variants of the int8 ferromagnet
 * (spin_set_variant: 0, 1, 3, 4 where supported) -- and, for a
 * double-checkerboard handle whose tile edge was left open (tile 0), every
 * supported tile edge (each gives its own chain, Sec. 3.2).  The fastest
 * choice is set on the handle and cached per (model, layout, dim, L,
 * lattices, order, hits, n_sweeps) for later handles of that shape.  Trials
 * run on the handle's buffer after a backup copy (allocated and freed by
 * this call); spins and counters are restored, so results do not depend on
 * whether or when the tuner ran.  best_variant, best_tile (host, optional)
 * receive the choice.  SPIN_EINVAL for bad arguments, SPIN_ENOMEM if the
 * backup cannot be allocated. */
int spin_tune(spin_lattice *lat, const void *couplings, const double *betas, int64_t n_sweeps,
              int32_t *best_variant, int32_t *best_tile);

const char *spin_strerror(int code);
void spin_destroy(spin_lattice *lat);

#ifdef __cplusplus
}
#endif
#endif /* SPIN_GB300_H */
