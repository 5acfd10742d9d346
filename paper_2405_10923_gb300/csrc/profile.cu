// Launch counting and per-phase CUDA-event timing (rhqr_profile_* in rhqr.h).
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rhqr {

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_profile_on{0};
static std::mutex g_mu;
struct Pending {
  int phase;
  cudaEvent_t a, b;
};
static std::vector<Pending> g_pending;
static double g_ms[PH_COUNT];
static long long g_calls[PH_COUNT];

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static std::atomic<int> g_last_cuda_error{0};
void note_cuda_error(cudaError_t e) { g_last_cuda_error.store((int)e, std::memory_order_relaxed); }

PhaseScope::PhaseScope(int ph, cudaStream_t s) : phase(ph), st(s), ev(nullptr) {
  if (!g_profile_on.load(std::memory_order_relaxed)) return;
  cudaEvent_t *e = new cudaEvent_t[2];
  if (cudaEventCreate(&e[0]) != cudaSuccess || cudaEventCreate(&e[1]) != cudaSuccess) {
    (void)cudaGetLastError();
    delete[] e;
    return;
  }
  cudaEventRecord(e[0], st);
  ev = e;
}

PhaseScope::~PhaseScope() {
  if (ev == nullptr) return;
  cudaEvent_t *e = (cudaEvent_t *)ev;
  cudaEventRecord(e[1], st);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back({phase, e[0], e[1]});
  delete[] e;
}

static void drain_pending() {
  for (auto &p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms[p.phase] += ms;
      g_calls[p.phase] += 1;
    } else {
      (void)cudaGetLastError();
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pending.clear();
}

}  // namespace rhqr

using namespace rhqr;

extern "C" {

int64_t rhqr_launch_count(void) { return g_launches.load(); }

int32_t rhqr_last_cuda_error(void) { return g_last_cuda_error.load(); }

const char *rhqr_cuda_error_name(int32_t code) { return cudaGetErrorName((cudaError_t)code); }

void rhqr_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_pending();
  for (int i = 0; i < PH_COUNT; ++i) {
    g_ms[i] = 0.0;
    g_calls[i] = 0;
  }
  g_profile_on.store(on ? 1 : 0);
}

int32_t rhqr_profile_read(double *ms, int64_t *calls, int32_t n) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_pending();
  int cnt = n < PH_COUNT ? n : PH_COUNT;
  for (int i = 0; i < cnt; ++i) {
    if (ms) ms[i] = g_ms[i];
    if (calls) calls[i] = g_calls[i];
  }
  return PH_COUNT;
}

}  // extern "C"
