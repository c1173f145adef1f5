// skei_fbp_noalloc: the FBP of skei_fbp for callers that cannot allocate
// device memory.  Its only scratch - the filtered sinogram - lives in a
// static device array of this library instead of a caller workspace.
#include "common.cuh"

// One array per GPU that loads the library, held until the process exits.
// Host code must not use the symbol as an address: it is a host-side
// stand-in; skei_fbp_noalloc looks the real device address up on the
// current device.
static __device__ __align__(256) float g_fbp_scratch[SKEI_FBP_NOALLOC_MAX_FLOATS];

namespace skei {
namespace {

constexpr double kPiNoAlloc = 3.14159265358979323846;

// Device address of g_fbp_scratch on the current device, with that device
// current.  It is looked up on every call: the lookup allocates nothing and
// is cheap once the module is loaded, and a cached address would go stale if
// the caller reset the device (cudaDeviceReset) and the array moved.  The
// first call on a device also loads the library's module there.
int scratch_address(float **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_fbp_scratch);
  if (e != cudaSuccess) return cuda_error(e, "skei_fbp_noalloc: cudaGetSymbolAddress");
  *out = static_cast<float *>(p);
  return SKEI_OK;
}

template <typename T>
int fbp_static(skei_plan p, const T *sino, int B, const int *idx, int m, T *x, float *scratch,
               cudaStream_t st) {
  // the filter writes every element of the B*m*n_det scratch that the
  // back-projection then reads, so nothing carried over from an earlier call
  // is ever used
  if (int rc = launch_filter<T, float>(p, sino, B * m, (float)(kPiNoAlloc / m), scratch, st))
    return rc;
  return launch_backproject<float, T, T>(p, scratch, B, idx, m, 1.0f, 0.0f, nullptr, x, st);
}

}  // namespace
}  // namespace skei

using namespace skei;

extern "C" int skei_fbp_noalloc(skei_plan plan, int dtype, const void *sino, int B,
                                const int *idx, int m, void *x, void *stream) {
  if (int rc = check_plan(plan)) return rc;
  if (int rc = check_dtype(dtype)) return rc;
  if (int rc = check_batch(B)) return rc;
  if (int rc = check_dev_ptr(sino, "sino")) return rc;
  if (int rc = check_dev_ptr(x, "x")) return rc;
  if (int rc = check_idx(plan, idx, m)) return rc;
  const size_t need = (size_t)B * m * plan->n_det;
  if (need > (size_t)SKEI_FBP_NOALLOC_MAX_FLOATS)
    return set_error(SKEI_EINVAL,
                     "skei_fbp_noalloc: B*m*n_det = %zu floats exceeds the static scratch of %d "
                     "floats; use skei_fbp with a workspace",
                     need, SKEI_FBP_NOALLOC_MAX_FLOATS);
  float *scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == SKEI_F32)
    return fbp_static<float>(plan, (const float *)sino, B, idx, m, (float *)x, scratch, st);
  return fbp_static<__nv_bfloat16>(plan, (const __nv_bfloat16 *)sino, B, idx, m,
                                   (__nv_bfloat16 *)x, scratch, st);
}
