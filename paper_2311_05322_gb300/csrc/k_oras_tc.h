// BF16 tensor-core (tcgen05) form of the ORAS apply (K4): layout plan and launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>

namespace mw {
struct Subdomains;
}

namespace mwk {
struct OrasTopo;
struct OrasBatch;

// Pre-tiled BF16 layout of the owned-row inverses W_s (see k_oras_tc.cu).
struct TcPlan {
  bool built = false;
  int n_sub = 0;
  int64_t n_mtiles = 0;       // sum_s ceil(n_own_s / 128)
  int64_t n_ktiles_total = 0; // sum_s ceil(2 n_s / 64)
  int64_t w_tiles = 0;        // sum_s mtiles_s * ktiles_s (16 KB each)
  // device arrays
  int32_t* mt_sub = nullptr;     // [n_mtiles] subdomain of each 128-row tile
  int32_t* mt_row0 = nullptr;    // [n_mtiles] first owned row
  int64_t* sub_wtile = nullptr;  // [n_sub] first W tile of s
  int64_t* sub_gtile = nullptr;  // [n_sub] first gathered-operand k tile of s
  int32_t* sub_kt = nullptr;     // [n_sub] k tiles of s
  int32_t* gt_sub = nullptr;     // [n_ktiles_total] subdomain of each gathered-operand tile
  int32_t* gt_kt = nullptr;      // [n_ktiles_total] its k tile
  int32_t* err = nullptr;        // device error word: nonzero after a timed-out wait
  int max_kt = 0;
};

bool tc_plan_build(TcPlan& p, const mw::Subdomains& sd, const std::function<void*(size_t)>& alloc, cudaStream_t s);
void tc_plan_free(TcPlan& p, const std::function<void(void*)>& dfree);
size_t tc_w_bytes(const TcPlan& p);
size_t tc_scratch_bytes(const TcPlan& p, int R);
void tc_extract(const TcPlan& p, const OrasBatch& bt, const OrasTopo& tp, int ws_prec, const void* ws, void* W,
                cudaStream_t s);
struct MfTask;
// Packs the FP32 blocks of tasks (A = src + a_off, [m][k], row stride lda, times the task's
// sign) into the plan's BF16 tiles for n plan "subdomains" that each stack up to two products
// with the same B (same k): subdomain q is task first[q] over task second[q] (rows of the second
// after those of the first; second[q] < 0: the first alone); ktmax / mtmax: the largest tile
// counts of the stacked products.
void tc_pack_stacked(const TcPlan& p, const MfTask* tasks, const int32_t* first, const int32_t* second, int n,
                     int ktmax, int mtmax, const float2* src, void* W, cudaStream_t s);
// stages: shared-memory pipeline depth of the MMA kernel (0 = default; the result does not depend
// on it, only the speed).  in_scale (may be null): per-column factor of r (z = M^{-1}(r * in_scale)).
// Output row q of "subdomain" s goes to z row own_glob[own_ptr[s] + q] (skipped when negative);
// c0_glob (may be null) lists, per output row, a row of z added to it (-1: none).  z_bf16: z is
// written as complex BF16 pairs (real in the low half), 4 bytes per value, row stride R values.
// persistent: CTAs loop over the output tiles with one copy ring and double-buffered
// accumulators (for plans of many short tiles; up to 64 columns, else the one-tile-per-CTA
// kernel runs); the same bits either way.
void oras_apply_tc(const TcPlan& p, const OrasTopo& tp, const void* W, const float2* r, float2* z, int R,
                   void* scratch, cudaStream_t s, int stages = 0, const double* in_scale = nullptr,
                   const int32_t* c0_glob = nullptr, bool z_bf16 = false, bool persistent = false);
// Pipeline depths the MMA kernel accepts for R columns: [tc_min_stages, tc_max_stages(R)].
constexpr int tc_min_stages = 2;
int tc_max_stages(int R);

// Launches the bounded-wait self-test (see k_oras_tc.cu); *code (device) gets 0 or 5.
void bounded_wait_probe(long long limit, int32_t* code, cudaStream_t s);

// Size of the fixed scratch used by mw_apply_preconditioner_noalloc (16 MiB).
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
// Device address of the fixed scratch on the current device (looked up once per device).
bool tc_noalloc_scratch(void** ptr, std::string& err);

}  // namespace mwk
