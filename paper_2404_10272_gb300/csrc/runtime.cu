// runtime.cu -- error reporting, version and the kernel profiler of the C ABI.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hdda_internal.cuh"

namespace hdda {

static thread_local char g_last_error[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  int code = (e == cudaErrorMemoryAllocation) ? HDDA_ERR_OOM : HDDA_ERR_CUDA;
  return set_error(code, "%s failed: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void clear_error() { g_last_error[0] = '\0'; }

// ---------------------------------------------------------------------------
// profiler
// ---------------------------------------------------------------------------
namespace {
struct ProfRecord {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;        // kernel timers
bool g_count_on = false;       // work counters
std::vector<ProfRecord> g_prof_records;
std::vector<cudaEvent_t> g_prof_pool;

cudaEvent_t take_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

bool profiler_on() {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  return g_prof_on;
}

bool counters_on() {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  return g_count_on;
}

namespace {
std::atomic<int> g_region_checks{0};
}  // namespace

bool region_checks_on() { return g_region_checks.load(std::memory_order_relaxed) != 0; }

namespace {
std::atomic<int> g_sampler_form{HDDA_SAMPLER_SEPARATE};
}  // namespace

int sampler_form() { return g_sampler_form.load(std::memory_order_relaxed); }

KernelTimer::KernelTimer(const char* name, cudaStream_t s, bool allow) : name_(name), s_(s) {
  if (!allow) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  if (!g_prof_on) return;
  a_ = take_event();
  if (a_ && cudaEventRecord(a_, s_) == cudaSuccess) live_ = true;
}

void KernelTimer::stop() {
  if (!live_) return;
  live_ = false;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  cudaEvent_t b = take_event();
  if (!b || cudaEventRecord(b, s_) != cudaSuccess) {
    g_prof_pool.push_back(a_);
    if (b) g_prof_pool.push_back(b);
    return;
  }
  g_prof_records.push_back(ProfRecord{name_, a_, b});
}

}  // namespace hdda

extern "C" const char* hdda_version(void) { return "hdda 0.1 (sm_103a)"; }

extern "C" const char* hdda_last_error(void) { return hdda::g_last_error; }

extern "C" int hdda_profiler_enable(int flags) {
  std::lock_guard<std::mutex> lock(hdda::g_prof_mu);
  hdda::g_prof_on = (flags & HDDA_PROFILE_TIMERS) != 0;
  hdda::g_count_on = (flags & HDDA_PROFILE_COUNTERS) != 0;
  return HDDA_OK;
}

extern "C" int hdda_set_region_checks(int on) {
  hdda::g_region_checks.store(on != 0, std::memory_order_relaxed);
  return HDDA_OK;
}

extern "C" int hdda_region_checks(void) { return hdda::region_checks_on() ? 1 : 0; }

extern "C" int hdda_set_sampler_form(int form) {
  if (form != HDDA_SAMPLER_FUSED && form != HDDA_SAMPLER_SEPARATE)
    return hdda::set_error(HDDA_ERR_INVALID_ARG, "sampler form %d is neither separate (0) "
                           "nor fused (1)", form);
  hdda::g_sampler_form.store(form, std::memory_order_relaxed);
  return HDDA_OK;
}

extern "C" int hdda_sampler_form(void) { return hdda::sampler_form(); }

extern "C" int hdda_profiler_read(hdda_kernel_time* out, int cap, int* n_out) {
  using namespace hdda;
  clear_error();
  std::lock_guard<std::mutex> lock(g_prof_mu);
  std::vector<std::string> names;
  std::vector<int64_t> launches;
  std::vector<double> ms;
  int status = HDDA_OK;
  for (const ProfRecord& r : g_prof_records) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && status == HDDA_OK) status = cuda_error(e, "profiler event");
    size_t i = 0;
    while (i < names.size() && names[i] != r.name) ++i;
    if (i == names.size()) {
      names.emplace_back(r.name);
      launches.push_back(0);
      ms.push_back(0.0);
    }
    launches[i] += 1;
    ms[i] += t;
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_records.clear();
  // work counters reported as pseudo-kernels (launches = count, no time)
  const unsigned long long evals[2] = {composite_take_blob_evals(), render_take_blob_evals()};
  const char* const eval_names[2] = {"composite_blob_evals", "render_blob_evals"};
  for (int i = 0; i < 2; ++i) {
    if (!evals[i]) continue;
    names.emplace_back(eval_names[i]);
    launches.push_back((int64_t)evals[i]);
    ms.push_back(0.0);
  }
  if (n_out) *n_out = (int)names.size();
  for (int i = 0; i < (int)names.size() && i < cap && out; ++i) {
    std::memset(&out[i], 0, sizeof(out[i]));
    std::strncpy(out[i].name, names[i].c_str(), sizeof(out[i].name) - 1);
    out[i].launches = launches[i];
    out[i].total_ms = ms[i];
  }
  return status;
}
