// The context behind the opaque p3m_sr_ctx handle.  Private to the library.
#pragma once

#include <string>

#include "common.cuh"

struct p3m_sr_ctx {
  p3m_sr_params prm{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  p3m::Geometry geo{};
  p3m::ForceConsts fc{};
  int64_t n = 0;                      // particles of the following calls (p3m_sr_set_count)
  int64_t cap = 0;                    // particles the scratch was allocated for (p3m_sr_create)
  int64_t n_tiles = 0;

  // ---- sort scratch ----
  int* keys[2] = {nullptr, nullptr};  // radix double buffers
  int* vals[2] = {nullptr, nullptr};
  int* offsets = nullptr;             // S + 1 (histogram, scanned in place)
  int64_t offsets_cap = 0;            // allocated ints of offsets
  int* cell = nullptr;                // sorted subtile ids (aliases keys[k])
  int* perm = nullptr;                // sorted -> input index (aliases vals[k])
  int* hist = nullptr;                // radix digit histograms
  int64_t hist_ints = 0;
  int* scan_scratch = nullptr;
  int64_t scan_scratch_ints = 0;
  void* gather_tmp = nullptr;         // 32 n bytes
  int radix_passes = 0;
  int radix_bits[4] = {0, 0, 0, 0};

  // ---- work lists ----
  int8_t* active_flag = nullptr;      // n
  int* act_scan = nullptr;            // n + 1
  int* active_idx = nullptr;          // n
  int* tile_chunks = nullptr;         // n_tiles + 1 (chunks per row segment, scanned)
  float4* part_acc = nullptr;         // partial sums of split chunks (work items x 32 lanes)
  p3m::Chunk* chunks = nullptr;       // receiver chunks of the last build_pairs
  p3m::Chunk* chunks_all = nullptr;   // chunks over all particles (vjp)
  int64_t max_chunks = 0;
  int* dev_small = nullptr;           // [0] n_chunks, [1] n_chunks_all, [2] n_active,
                                      // [3..7] work counters
  unsigned long long* pair_count = nullptr;

  // ---- per-call arrays ----
  float4* rel4 = nullptr;             // FP32 subtile-relative coordinates (+ id bits)
  double* org = nullptr;              // subtile origins per axis (geo.org points here)
  int64_t org_cap = 0;                // allocated doubles of org
  float4* abar4 = nullptr;            // vjp: masked abar, FP32
  double* abar_d = nullptr;           // vjp: masked abar, FP64 (3 n)
  float* table = nullptr;             // tabulated bracket (p3m_sr_forces_tabulated)
  int table_bits = 0;

  // ---- error latch ----
  int* err_dev = nullptr;
  int* err_host = nullptr;            // pinned mirror
  cudaEvent_t err_event = nullptr;
  bool err_event_pending = false;

  // ---- instrumentation ----
  int64_t launches = 0;               // kernels launched by this context (cumulative)
  cudaEvent_t kt_ev[4] = {nullptr, nullptr, nullptr, nullptr};  // traversal kernel brackets (fwd, vjp)
  bool kt_pending[2] = {false, false};
  double kt_ms[2] = {0.0, 0.0};       // last forward / vjp traversal kernel time

  // ---- state ----
  bool sorted = false;
  const double* sorted_pos = nullptr;  // array sorted by the last p3m_sr_sort (rel4 matches it)
  float* drift_slots = nullptr;        // kMaxDrifts: largest displacement of each drift since the sort
  int n_drift = 0;                     // drifts applied to sorted_pos since the sort
  bool rel4_stale = false;             // sorted_pos moved after rel4 was written
  bool pairs_built = false;
  bool all_chunks_built = false;
  bool all_active = true;
  bool symmetric = true;               // all-active FP32 forces: each pair once, both updated

  std::string last_error;
};

namespace p3m {

// Set the context's message and return the status.
p3m_status fail(p3m_sr_ctx* ctx, p3m_status st, const std::string& msg);
// Check a CUDA call; on failure set the message and return P3M_ERR_CUDA.
p3m_status cuda_check(p3m_sr_ctx* ctx, cudaError_t e, const char* what);
// Return a latched device error (if a previous report has landed), else P3M_OK.
p3m_status poll_latched(p3m_sr_ctx* ctx);
// Enqueue the copy of the device error word to the pinned mirror.
void report_latched(p3m_sr_ctx* ctx);
// Build (if needed) the chunk list over all particles.
p3m_status ensure_all_chunks(p3m_sr_ctx* ctx);

}  // namespace p3m

// Parameter checks and derived constants of p3m_sr_create (host.cu).
p3m_status validate_params(p3m_sr_ctx* ctx, const p3m_sr_params& p);
void setup_geometry(p3m_sr_ctx* ctx);
void setup_force_consts(p3m_sr_ctx* ctx);
