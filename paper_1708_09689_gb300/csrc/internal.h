// Host-side internals shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdlib>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pvsc.h"
#include "common.cuh"

namespace pvsc {

int set_error(int code, const char* fmt, ...);
inline int ok() { return PVSC_OK; }

#define PVSC_CUDA_TRY(call)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return ::pvsc::set_error(PVSC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Launch shape of one sweep kind on one lattice.
struct LaunchShape {
  int threads = 256;
  int blocks_per_sm = 0;  // 0: occupancy maximum
  int zslab = 0;          // 0: automatic
  int vpt = 0;            // 0: automatic
  int tile_x = 0;         // > 0: shared-memory staged TI sweep with this tile
  int tile_y = 0;
  int kernel = 0;         // TI: 0 z-marching / staged, 1 flat, 2 / 3 cp.async rings,
                          // 4 two KPM steps per sweep (tile_x x tile_y tiles),
                          // 5 z-marching over tile_x x tile_y column tiles, 6 marching along x,
                          // 7 TMA-staged plane tiles (warp-specialised)
};

// kernel-selector "model" values of the flat and the cp.async-prefetching TI
// sweeps in the launch tables
constexpr int kModelTIFlat = 3;
constexpr int kModelTIAsync = 4;      // ring of all six blocks of a plane, one plane ahead
constexpr int kModelTIAsyncDeep = 5;  // ring of the two HBM streams, three planes ahead
constexpr int kModelWSM = 8;         // Weyl semimetal flat cell sweep
constexpr int kModelWSMMarch = 9;    // Weyl semimetal z-marching cell sweep
constexpr int kModelGrapheneQD = 10; // graphene sweep with the regenerated quantum-dot array
constexpr int kModelTIXMarch = 11;   // TI sweep marching along x (tuning kernel 6)
constexpr int kModelTIFx = 12;       // TI KPM sweep on fixed-point (PVSC_Q64) vectors
constexpr int kAsyncDepth = 1;
constexpr int kAsyncDeepDepth = 3;
// ring: (depth + 1) slots x buffers x 4 granules of 16 bytes per thread
inline size_t async_ring_bytes(int model, int threads) {
  if (model == kModelTIAsync) return (size_t)(kAsyncDepth + 1) * 6 * 4 * threads * 16;
  if (model == kModelTIAsyncDeep) return (size_t)(kAsyncDeepDepth + 1) * 2 * 4 * threads * 16;
  return 0;
}
int allow_max_smem(void* fn);

// shared-memory staged TI sweep (sweep_c128.cu / sweep_c64.cu)
int launch_sweep_bulk(int prec, int feat, int grid, int threads, size_t smem, const Sweep& p,
                      cudaStream_t st);
int launch_sweep_bulk_c128(int feat, int grid, int threads, size_t smem, const Sweep& p,
                           cudaStream_t st);
int launch_sweep_bulk_c64(int feat, int grid, int threads, size_t smem, const Sweep& p,
                          cudaStream_t st);
int occupancy_bulk_c128(int feat, int threads, size_t smem, int* blocks);
int occupancy_bulk_c64(int feat, int threads, size_t smem, int* blocks);
int bulk_error_c128(int clear, int* flag);
int bulk_error_c64(int clear, int* flag);
int occupancy_bulk(int prec, int feat, int threads, size_t smem, int* blocks);
int bulk_sweep_error(int prec, int clear, int* flag);
size_t bulk_smem_bytes(int TX, int TY, int R, int prec);

// fixed-point KPM (sweep_fx.cu): work layout (byte offsets) and launchers
struct FxLayout {
  int nb;
  size_t part, xscale, vscale, dfx, wa, wb, total;
};
FxLayout fx_layout(const pvsc_lattice* lat, int R);
int launch_fx_prepare(const pvsc_lattice* lat, int R, const void* r0, uint64_t seed, double a,
                      double b, void* work, const FxLayout& L, cudaStream_t st);
int launch_sweep_fx(const pvsc_lattice* lat, Sweep& p, const LaunchShape& sh, bool tuned,
                    cudaStream_t st);

// two KPM recurrence steps per sweep (sweep_kpm2.cu): complex64 TI lattices, R >= 2
constexpr int kKernelKpm2 = 4;
// z-marching TI sweep over 2D column tiles (tile_x x tile_y columns per block)
constexpr int kKernelTiles = 5;
// TI sweep marching along x instead of z (short z extents)
constexpr int kKernelXMarch = 6;
// TI (and Weyl-cell) sweep with TMA-staged z-plane tiles (sweep_tma.cu):
// complex64, R = 4 .. 64, Lx a multiple of 4
constexpr int kKernelTma = 7;
bool tma_sweep_possible(const pvsc_lattice* lat, int R, int prec);
int launch_sweep_tma(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
// the same tiles marching along x (tiles over (y, z) columns): TI, complex64; the
// fused step with z falls back to kernel 7
constexpr int kKernelTmaX = 8;
bool tma_xm_possible(const pvsc_lattice* lat, int R, int prec);
int launch_sweep_tma_xm(const pvsc_lattice* lat, int feat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int tma_error(int clear, int* flag);
// fixed-point (PVSC_Q64) KPM sweep on TMA-staged tiles (sweep_tma_fx.cu)
bool tma_fx_possible(const pvsc_lattice* lat, int R);
int launch_sweep_tma_fx(const pvsc_lattice* lat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int tma_error_fx(int clear, int* flag);
bool tma_tile_valid(int R, int tile_x, int tile_y);  // (0, 0) or one of the two tiles of this R
bool tma_tile_deep(int R, int tile_y);
int launch_kpm2_sweep(const pvsc_lattice* lat, Sweep& p, const LaunchShape& sh, cudaStream_t st);
int kpm2_check_tile(int TX, int TY, int R);

// Vectors per thread for (R, prec) under an optional tuned value.
int vpt_tuned(int tuned, int R, int prec);

struct Graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace pvsc

struct pvsc_lattice;
namespace pvsc {
template <class F>
int run_graph(const pvsc_lattice* clat, const std::vector<uint64_t>& key, cudaStream_t st, F&& body);
}

struct pvsc_lattice {
  pvsc::Geometry g{};
  double* V_dev = nullptr;  // owned when v_mode == 1
  float* V32_dev = nullptr; // fp32 copy of V_dev for complex64 sweeps
  pvsc::QDots* qd_dev = nullptr;  // quantum-dot array parameters (v_mode 3)
  pvsc::QDScal qds{};             // and the scalars the sweeps take as parameters
  int v_source = 0;
  uint64_t seed = 0;
  int device = 0;
  int sm_count = 0;
  std::map<std::pair<int, int>, pvsc_tuning> tuning;  // (R, prec) -> tuning
  // cached CUDA graphs keyed by the full argument set of a captured loop
  std::map<std::vector<uint64_t>, pvsc::Graph> graphs;
  // Process-unique stamp of the lattice's state, renewed whenever its cached
  // graphs go stale (creation, new potential, new tuning): graphs that capture
  // other lattices' geometry (the batched KPM) key on it, so that a changed
  // potential or a new lattice at a reused address never replays old arguments.
  uint64_t generation = 0;
  // exact Gershgorin interval of H, kept once computed (the fixed-point KPM
  // checks its scaling against it); cleared when the potential changes
  bool gersh_valid = false;
  double gersh_lo = 0.0, gersh_hi = 0.0;
  std::mutex mu;
  ~pvsc_lattice();
};

namespace pvsc {

constexpr int kMaxGridPerSM = 16;
constexpr size_t kWorkHeader = 256;  // counters at the start of every work buffer

int vpt_for(int R, int prec);
bool valid_R(int R);
int check_lattice(const pvsc_lattice* lat);
int check_ptr(const void* p, const char* name);

// Fill p.g / p.R / p.C from the lattice; the caller sets the rest.
void sweep_init(Sweep& p, const pvsc_lattice* lat, int R, int prec);
// Launch one fused sweep (feat: F_* mask).  Dot features need p.partials and
// p.counter inside a work buffer of at least dots_work_bytes(lat, R) bytes.
int launch_sweep(const pvsc_lattice* lat, int prec, int feat, Sweep& p, cudaStream_t st);
int launch_sweep_shape(const pvsc_lattice* lat, int prec, int feat, Sweep& p, LaunchShape sh, cudaStream_t st);
int kpm_enqueue(const pvsc_lattice* lat, int R, int prec, const void* r0, uint64_t seed, int M, double a,
                double b, double* mu, void* work, const LaunchShape* force, cudaStream_t cs);
size_t dots_work_bytes(const pvsc_lattice* lat, int R);
size_t vec_bytes(const pvsc_lattice* lat, int R, int prec);  // one D x R block

// per-precision kernel launchers (sweep_c128.cu / sweep_c64.cu)
int launch_sweep_c128(int model, int feat, int grid, int threads, const Sweep& p,
                      cudaStream_t st);
int launch_sweep_c64(int model, int vpt, int feat, int grid, int threads, const Sweep& p,
                     cudaStream_t st);
int occupancy_c128(int model, int feat, int threads, int* blocks);
int occupancy_c64(int model, int vpt, int feat, int threads, int* blocks);

// elementwise helpers (aux.cu)
int launch_random_phase(void* out, int prec, int64_t D, int R, uint64_t seed, cudaStream_t st);
int launch_convert_c128_to_c64(const void* in, void* out, int64_t n, cudaStream_t st);
int launch_scale_init(const void* x128, double2* acc, double cr, double ci, int64_t n,
                      cudaStream_t st);
int launch_seed_potential(double* V, int64_t n, uint64_t seed, double W, cudaStream_t st);
int launch_get_potential(const Geometry& g, double* out, cudaStream_t st);
int launch_potential_f32(const double* V, float* V32, int64_t n, cudaStream_t st);
int launch_gershgorin(const Geometry& g, double* out, int grid, cudaStream_t st);
int launch_neighbours(const Geometry& g, int64_t* nbr, cudaStream_t st);
int launch_adjoint_top(const pvsc_lattice* lat, int R, const double2* G, double sr, double si,
                       double2* uM, const double2* w, double gscale, double* grad,
                       cudaStream_t st);

// ---------------------------------------------------------------- CUDA graph cache
// Drop every cached graph of the lattice: a graph holds the launch shapes and
// kernel arguments it was captured with, so a new tuning or a new potential
// mode makes it stale.
inline uint64_t next_generation() {
  static std::atomic<uint64_t> counter{0};
  return ++counter;
}

inline void drop_graphs(pvsc_lattice* lat) {
  std::lock_guard<std::mutex> lk(lat->mu);
  lat->generation = next_generation();
  for (auto& kv : lat->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  lat->graphs.clear();
}

// Programmatic dependent launch of the TMA-staged sweeps (on unless
// PVSC_NO_PDL is set to a value other than 0).
inline bool pdl_enabled() {
  const char* e = std::getenv("PVSC_NO_PDL");
  return !(e && e[0] && e[0] != '0');
}

inline bool graphs_enabled() {
  const char* e = std::getenv("PVSC_NO_GRAPH");
  return !(e && e[0] && e[0] != '0');
}

template <class F>
int run_graph(const pvsc_lattice* clat, const std::vector<uint64_t>& key, cudaStream_t st,
                     F&& body) {
  if (!graphs_enabled()) return body(st);
  pvsc_lattice* lat = const_cast<pvsc_lattice*>(clat);
  std::lock_guard<std::mutex> lk(lat->mu);
  auto it = lat->graphs.find(key);
  if (it == lat->graphs.end()) {
    if (lat->graphs.size() >= 32) {
      for (auto& kv : lat->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
      }
      lat->graphs.clear();
    }
    cudaStream_t cs;
    PVSC_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cs);
      return set_error(PVSC_ERR_CUDA, "graph capture failed to start: %s", cudaGetErrorString(e));
    }
    const int rc = body(cs);
    Graph gr;
    e = cudaStreamEndCapture(cs, &gr.graph);
    cudaStreamDestroy(cs);
    if (rc == PVSC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&gr.exec, gr.graph, 0);
    if (rc != PVSC_OK || e != cudaSuccess) {
      // a launch the capture did not accept: run the same launches directly
      if (gr.graph) cudaGraphDestroy(gr.graph);
      cudaGetLastError();
      return body(st);
    }
    it = lat->graphs.emplace(key, gr).first;
  }
  PVSC_CUDA_TRY(cudaGraphLaunch(it->second.exec, st));
  return PVSC_OK;
}

}  // namespace pvsc
