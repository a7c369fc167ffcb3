// fv_tune.cu -- lookup in the kernel-choice table recorded by the autotuner.
#include <cstdio>

#include "fv_tune.h"

namespace fv {

static const TuneEntry kTuneTable[] = {
#include "fv_tune_table.inc"
    {-1, -1, -1, -1, nullptr, 0.0, nullptr},  // end of the table
};

int tune_size_class(long long cells) {
  if (cells < (1LL << 16)) return 0;
  if (cells < (1LL << 20)) return 1;
  if (cells < (1LL << 24)) return 2;
  return 3;
}

const TuneEntry *tune_lookup(int system, int precision, long long cells, int mode) {
  const int k = tune_size_class(cells);
  for (const TuneEntry *e = kTuneTable; e->kernel; ++e)
    if (e->system == system && e->precision == precision && e->size_class == k && e->mode == mode) return e;
  return nullptr;
}

std::string tune_describe(const TuneEntry &e) {
  static const char *sys[] = {"advection", "euler", "spray"};
  static const char *prec[] = {"f64", "f32", "bf16"};
  static const char *mode[] = {"two-buffer", "in-place", "two-step", "batched"};
  char buf[256];
  std::snprintf(buf, sizeof(buf), "table: %s %s %s class %d (%s, %.4g G cell-updates/s when recorded)",
                (e.system >= 0 && e.system < 3) ? sys[e.system] : "?",
                (e.precision >= 0 && e.precision < 3) ? prec[e.precision] : "?",
                (e.mode >= 0 && e.mode < 4) ? mode[e.mode] : "?", e.size_class, e.workload, e.rate / 1e9);
  return buf;
}

}  // namespace fv
