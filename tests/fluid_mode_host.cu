// Host harness for the CUDA library's per-mode fluid response (the
// __host__ __device__ function k_fluid_table evaluates per mode), used by
// tests/test_fluid_mode_host.py on a machine without a GPU: prints
// kappa g_T g_L for eps, z0 and the kappas given on the command line.
#include "../paper_1908_04279_gb300/csrc/mm_fluid.cu"

#include <cstdio>
#include <cstdlib>

// The solve entry points of mm_fluid.cu call these; the harness never does.
namespace mmh {
mm_status run_moments(mm_handle*) { return MM_ERR_UNSUPPORTED; }
mm_status velocity_update(mm_handle*) { return MM_ERR_UNSUPPORTED; }
mm_status check_status(mm_handle*) { return MM_ERR_UNSUPPORTED; }
}  // namespace mmh

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  const double eps = atof(argv[1]), z0 = atof(argv[2]);
  for (int i = 3; i < argc; ++i) {
    const double k = atof(argv[i]);
    const double2 g = mm::fl_mode_response(k, eps, z0);
    printf("%.17g %.17g %.17g\n", k, g.x, g.y);
  }
  return 0;
}
