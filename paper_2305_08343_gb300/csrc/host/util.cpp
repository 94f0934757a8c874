// util.cpp — errors, threads and timing for the host side of libsubcull.
#include <atomic>
#include <chrono>
#include <exception>
#include <cstdarg>
#include <cstdio>
#include <thread>

#include "internal.h"

namespace sc {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

const char* last_error_cstr() { return g_last_error.c_str(); }

void fail(sc_status code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  throw Error{code, buf};
}

int resolve_threads(int requested) {
  int hw = (int)std::thread::hardware_concurrency();
  if (hw <= 0) hw = 1;
  if (requested <= 0) return hw;
  return requested < hw * 4 ? requested : hw * 4;
}

void parallel_for(int64_t n, int threads, int64_t grain,
                  const std::function<void(int64_t)>& fn) {
  if (n <= 0) return;
  if (grain < 1) grain = 1;
  int64_t blocks = (n + grain - 1) / grain;
  int t = threads;
  if (t > blocks) t = (int)blocks;
  if (t <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> pool;
  std::exception_ptr err = nullptr;
  std::atomic<bool> failed{false};
  auto work = [&]() {
    try {
      for (;;) {
        int64_t blk = next.fetch_add(1);
        if (blk >= blocks || failed.load()) break;
        int64_t e = (blk + 1) * grain < n ? (blk + 1) * grain : n;
        for (int64_t i = blk * grain; i < e; ++i) fn(i);
      }
    } catch (...) {
      if (!failed.exchange(true)) err = std::current_exception();
    }
  };
  for (int i = 0; i < t - 1; ++i) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

void parallel_ranges(int64_t n, int parts,
                     const std::function<void(int64_t, int64_t, int)>& fn) {
  if (parts < 1) parts = 1;
  if (parts == 1 || n < 2 * parts) {
    fn(0, n, 0);
    return;
  }
  std::vector<std::thread> pool;
  for (int p = 1; p < parts; ++p)
    pool.emplace_back([&, p]() { fn(n * p / parts, n * (p + 1) / parts, p); });
  fn(0, n / parts, 0);
  for (auto& th : pool) th.join();
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace sc
