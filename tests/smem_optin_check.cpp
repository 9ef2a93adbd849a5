// Host-only check of dfacto::SmemOptIn (csrc/smem_optin.h): the shared memory
// opt-in is tracked per (kernel, device), so a second device gets its own
// call, a size already covered makes none, and a failed call is retried.
// Prints one line per check; exits non-zero on the first failure.
#include <cstdio>
#include <thread>
#include <vector>

#include "smem_optin.h"

static int fails = 0;
#define CHECK(cond)                                                   \
  do {                                                                \
    if (!(cond)) {                                                    \
      std::printf("FAIL line %d: %s\n", __LINE__, #cond);             \
      ++fails;                                                        \
    } else {                                                          \
      std::printf("ok: %s\n", #cond);                                 \
    }                                                                 \
  } while (0)

int main() {
  dfacto::SmemOptIn t;
  int kernel_a = 0, kernel_b = 0;  // stand-ins for two kernels' addresses
  const void* ka = &kernel_a;
  const void* kb = &kernel_b;
  std::vector<int> calls;  // device of every set() that ran
  auto set_on = [&](int dev, int result) {
    return [&calls, dev, result] { calls.push_back(dev); return result; };
  };

  CHECK(t.ensure(ka, 0, 64 << 10, set_on(0, 0)) == 0);
  CHECK(calls.size() == 1);
  // same kernel, same device, same or smaller size: no call
  CHECK(t.ensure(ka, 0, 64 << 10, set_on(0, 0)) == 0);
  CHECK(t.ensure(ka, 0, 50 << 10, set_on(0, 0)) == 0);
  CHECK(calls.size() == 1);
  // the same kernel on a second device needs its own call
  CHECK(t.ensure(ka, 1, 64 << 10, set_on(1, 0)) == 0);
  CHECK(calls.size() == 2 && calls[1] == 1);
  // a larger size on device 0 calls again; device 1 keeps its own record
  CHECK(t.ensure(ka, 0, 96 << 10, set_on(0, 0)) == 0);
  CHECK(calls.size() == 3 && calls[2] == 0);
  CHECK(t.ensure(ka, 1, 96 << 10, set_on(1, 0)) == 0);
  CHECK(calls.size() == 4 && calls[3] == 1);
  // another kernel on device 0 is tracked apart
  CHECK(t.ensure(kb, 0, 64 << 10, set_on(0, 0)) == 0);
  CHECK(calls.size() == 5);
  // a failing set() is reported and not remembered: the next call tries again
  CHECK(t.ensure(kb, 2, 64 << 10, set_on(2, 7)) == 7);
  CHECK(t.ensure(kb, 2, 64 << 10, set_on(2, 0)) == 0);
  CHECK(calls.size() == 7);
  // many threads asking for one (kernel, device, size): exactly one call
  dfacto::SmemOptIn u;
  int count = 0;
  std::vector<std::thread> th;
  for (int i = 0; i < 8; ++i)
    th.emplace_back([&] {
      for (int j = 0; j < 1000; ++j) u.ensure(ka, 3, 80 << 10, [&] { ++count; return 0; });
    });
  for (auto& x : th) x.join();
  CHECK(count == 1);
  std::printf(fails ? "FAILED %d\n" : "ALL OK\n", fails);
  return fails ? 1 : 0;
}
