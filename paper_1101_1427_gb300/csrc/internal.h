// Host-side handle and the launchers each translation unit provides.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/spin.h"
#include "common.cuh"

// NVTX range over one ABI call, so that a profiler's timeline shows which
// entry point enqueued which kernels (no cost when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

namespace spin {
// Decomposition of the resident 3D Heisenberg sweeps (heis_res.cu).
struct HeisResPlan {
  int Py, Pz;   // pencils per lattice along y and z
  int grid;     // CTAs: n_lat Py Pz, one per SM at most
  size_t smem;  // dynamic shared memory per CTA
};
}  // namespace spin

struct spin_lattice {
  spin_desc d;
  spin::Geom g;
  cudaStream_t stream;
  void *spins;           // caller-owned
  void *couplings;       // caller-owned (may be NULL)
  int64_t n_lat;         // n_sets * n_temps * n_real lattices
  int64_t sweeps_done;
  int64_t pt_steps_done;
  int variant;           // 2D int8 sweep: 0 phases, 1 fused
  int msc_width;         // EA coded: realisations sharing one uniform (32 or 64)
  int order;             // spin_update_order
  int order_tile;        // double checkerboard: tile edge T
  int order_hits;        // double checkerboard: hits k per compound move

  // handle-owned device workspaces
  uint32_t *d_thr;       // [n_temps][4] Metropolis thresholds, index dE/4
  std::vector<double> betas_cached;
  int thr_valid;
  uint32_t *d_pt_thr;    // concatenated replica-exchange tables
  int32_t *d_pt_off;     // [n_temps]: offset of pair t's table
  int32_t *d_pt_len;     // [n_temps]: its length (entries beyond are 0)
  double *d_pt_dbeta;    // [n_temps]: beta_{t+1} - beta_t
  std::vector<double> pt_betas_cached;
  int64_t *d_energy;     // [n_lat] scratch energies for the exchange step
  int64_t *d_scratch64;  // small reduction scratch
  int *d_err;            // device error word
  void *d_pingpong;      // lattice-sized buffer of the fused 2D sweep (lazy)
  size_t pingpong_bytes;
  // batched launches (options set with spin_set_batch_options)
  uint64_t batch_timeout_ns;  // bound on every team-barrier wait (0: 2 s)
  int batch_ctas_per_sm;      // 0: autotuned / default
  double batch_ising_scale;   // 0: autotuned / default; weight of Ising units in the CTA split
  double batch_ea_n0;         // 0: autotuned / default; else 1 + fixed cost per EA word-lattice, in sites
  int batch_fault_extra;      // arrivals a barrier waits for that never come (tests)
  // batched-launch workspace, allocated by the first uncaptured batch call
  int64_t *d_ctr;             // [sweeps_done, pt_steps_done] as the batch kernel reads them
  unsigned *d_bar;            // one team-barrier counter per work unit of this handle
  int *d_escr;                // EA: [group][n_sets][n_temps][32] energy scratch
  int64_t ctr_dev[2];         // what d_ctr holds once the enqueued work is done (-1: unknown)
  // resident 3D Heisenberg sweeps (heis_res.cu), allocated on first use
  unsigned *d_res_flags;      // one published-phase counter per CTA
  int res_flags_n;
  uint32_t res_base;          // phases the counters have advanced by in earlier launches
  spin::HeisResPlan res_plan[2];  // per variant (full accuracy, fast math)
  int res_plan_state[2];          // 0: not made yet, 1: usable, -1: the lattices do not fit
};

namespace spin {

// ising_i8.cu
cudaError_t launch_init_i8(spin_lattice *h);
cudaError_t launch_couplings_i8(spin_lattice *h);
cudaError_t launch_sweeps_i8(spin_lattice *h, const int8_t *J, int64_t n_sweeps);

// msc.cu
cudaError_t launch_init_msc(spin_lattice *h);
cudaError_t launch_couplings_msc(spin_lattice *h);
cudaError_t launch_sweeps_msc(spin_lattice *h, const uint32_t *J, int64_t n_sweeps);
cudaError_t launch_unpack_msc(spin_lattice *h, int8_t *out);
cudaError_t launch_pack_msc(spin_lattice *h, const int8_t *in);

// heis.cu
cudaError_t launch_init_heis(spin_lattice *h);
cudaError_t launch_sweeps_heis(spin_lattice *h, int64_t n_sweeps);

// heis_res.cu: 3D lattices resident in the SMs' shared memory for a whole
// call, one pencil of rows per CTA (L = 64 or 128, where they fit); the
// plan (HeisResPlan, above the handle) is made once per handle and variant
bool heis_resident_plan(const spin_lattice *h, HeisResPlan *plan);
// sweeps sweep0 .. sweep0 + n_sweeps - 1 (no renormalisation inside)
cudaError_t launch_sweeps_heis_resident(spin_lattice *h, const HeisResPlan &plan, int64_t sweep0, int64_t n_sweeps);

// measure.cu
cudaError_t launch_measure(spin_lattice *h, const void *J, int64_t *E, int64_t *M, int64_t *Q,
                           double *Ef, double *Mf);
// energies: the lattices' current energies if the caller has them (device,
// [n_lat]), else NULL to compute them
// labels: configuration labels moved with accepted exchanges (device, [n_lat], or NULL)
cudaError_t launch_pt_swap(spin_lattice *h, const void *J, int64_t *accepted, int32_t *labels,
                           const int64_t *energies);

// Launches kernel k as a programmatic dependent of the previous work in
// stream s (the kernel must call griddep_wait() before touching memory).
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// rng.cu
cudaError_t launch_rng_fill(uint64_t seed, uint32_t w, uint32_t lattice_id, uint32_t sweep,
                            uint64_t count, uint32_t *out, cudaStream_t s);
cudaError_t launch_rng_probe(uint64_t seed, uint32_t threads, uint32_t calls, uint32_t *out,
                             cudaStream_t s);

// probe.cu (returns a SPIN_* status)
int launch_pipe_probe(int op, int blocks_per_sm, uint32_t iters, long long *clocks, uint32_t *sink,
                      int *sms, cudaStream_t s);

// heis.cu (double checkerboard of the 2D Heisenberg model)
cudaError_t launch_heis_dcb_tiles(spin_lattice *h, int coarse, uint32_t sweep0);
cudaError_t launch_heis_renorm(spin_lattice *h);

// ising_i8.cu: whole-lattice-in-shared-memory sweeps of small 2D and 3D
// int8 ferromagnets (variant 3)
constexpr int kResidentMaxL = 128;  // 2D
constexpr int kResident3MaxL = 24;  // 3D (four chunks per thread of 512)
bool resident_supported(int dim, int L);
// n sweeps; with E or M (device, rows of n_lat) also measures after the
// sweeps first, first + every, ... (1-based in the call) into rows 0, 1, ...
cudaError_t launch_resident(spin_lattice *h, int64_t n_sweeps, int64_t *E, int64_t *M, int every, int first);

// dcb.cu
bool dcb_supported(const spin_lattice *h, int tile);
cudaError_t launch_sweeps_dcb(spin_lattice *h, int64_t n_sweeps);

// batch.cu: load the batch kernel's device counters from the host counters
int sync_device_counters(spin_lattice *h, cudaStream_t st);

inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace spin
