// fv_tune.h -- the kernel-choice table the autotuner records.
//
// For every (system, precision, grid-size class, mode) it measured, the
// autotuner (python -m paper_1701_05431_gb300.autotune, on the GPU) times
// every compiled kernel candidate on a seeded workload of that class with
// CUDA events and records the fastest in fv_tune_table.inc, which this
// library compiles in.  A context created with fv_config.tune = 0 takes the
// recorded candidate for its key; keys the table lacks fall back to the
// occupancy heuristic of the host code.
#pragma once

#include <string>

namespace fv {

// How a kernel is used: two state buffers, one buffer updated in place, two
// time steps per launch, or the batched persistent launch.
enum TuneMode { kTuneSingle = 0, kTuneInplace = 1, kTuneTwoStep = 2, kTuneBatch = 3 };

struct TuneEntry {
  int system;        // kAdvection / kEuler / kSpray
  int precision;     // 0 f64, 1 f32, 2 bf16 storage
  int size_class;    // tune_size_class of the cell count
  int mode;          // TuneMode
  const char *kernel;    // candidate description (as fv_kernel_candidate lists it)
  double rate;           // its measured cell-updates/s
  const char *workload;  // the workload it was measured on
};

// Grid-size class of a cell count (for a batch: the cells of all instances):
// 0 below 2^16 cells, 1 below 2^20, 2 below 2^24, 3 from 2^24 on.
int tune_size_class(long long cells);

// The recorded entry for this key, or nullptr.
const TuneEntry *tune_lookup(int system, int precision, long long cells, int mode);

// "table: <system> <precision> <mode> class <k> (<workload>, <rate> G
// cell-updates/s when recorded)" for an entry.
std::string tune_describe(const TuneEntry &e);

}  // namespace fv
