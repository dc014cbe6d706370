// model.h -- the opaque qcl_model handle (host copy of the model and its
// device constant block), shared by the translation units of the C ABI.
#pragma once
#include <string>
#include <vector>

#include "qcl_common.cuh"

struct qcl_model {
  int ns = 0, n = 0;
  double hbar = 1.0, hop_scale = 1.0, p_max = 0.5;
  std::vector<double> mass, omega, E, K;
  qcl::DevModel host{};
  qcl::DevModel* dev = nullptr;  // device block: DevModel followed by K
  int device = 0;
  // launch shape of the FP32-bulk kernels (qcl_set_launch_shape / qcl_autotune;
  // 0 = default)
  int shape_wpt = 0, shape_bps = 0;
  int shape_outs = 0;  // output times per persistent launch (0 = kChunkOut)
  double shape_rate = 0.0;
};

namespace qcl {
// Records `msg` as the calling thread's last error and returns `st`.
qcl_status set_error(qcl_status st, const char* msg);
// The ensemble-descriptor checks every entry point makes (message recorded).
qcl_status check_ensemble(const qcl_model* m, const qcl_ensemble_desc* e);
// The process-wide QCL_OPT_GRID_CAP value.
int64_t option_grid_cap();
// The process-wide QCL_OPT_MODES_IN_MEMORY value (0, 1 or 2).
int option_modes_in_memory();
}  // namespace qcl
