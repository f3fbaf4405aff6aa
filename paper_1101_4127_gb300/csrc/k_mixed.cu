// k_mixed.cu -- mixed-precision transport (FP32 traversal and attenuation,
// int64 deposits).  Placeholder until the kernels land.
#include "crash_internal.cuh"

int launch_trace_mixed(const StepArgs&, const BinTables&, const crash_run_opts&, void*,
                       cudaStream_t, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>*, int*) {
  return -1;
}
void* wavefront_create(int64_t, int64_t, int, int* status) {
  static int dummy;
  *status = 0;
  return &dummy;
}
void wavefront_destroy(void*) {}
int64_t wavefront_capacity(void*) { return 0; }
