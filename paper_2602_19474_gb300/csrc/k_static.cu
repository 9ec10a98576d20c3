// k_static.cu -- boundary extraction into caller buffers without any device
// allocation.
//
// mesh_bitmap allocates its working memory from the CUDA stream-ordered
// allocator.  Some callers cannot do that: a host application that hands the
// library a fixed device budget and forbids it from allocating, or a caller
// on a latency-critical path where an allocation may block or fail under
// memory pressure.  sbmt_extract_segments_static serves them for the first
// step of the path (the pixel-edge boundary runs): its only working memory is
// the file-scope array below, reserved when the library is loaded and kept
// by every device that loads it until the process exits.
#include <cstdio>
#include <mutex>

#include "sbmt.h"
#include "sbmt_launch.h"

using namespace sbmt;

namespace {

// working memory of the no-allocation path: 4 words of counters, then the
// two corner bit-planes (row-packed and column-packed)
constexpr size_t kStaticWords = (size_t)1 << 21;  // 8 MiB
static __device__ __align__(256) unsigned int g_static_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned int* g_static_ptr[kMaxDevices] = {};

thread_local char g_static_err[256];

__global__ void k_static_count(const u32* nseg, const u32* err, u32* d_count) {
  if (threadIdx.x == 0) *d_count = *err ? NONE : *nseg;
}

int static_fail(int code, const char* msg) {
  std::snprintf(g_static_err, sizeof g_static_err, "%s", msg);
  return code;
}

}  // namespace

extern "C" const char* sbmt_static_last_error(void) { return g_static_err; }

extern "C" int sbmt_extract_segments_static(const void* d_image, int32_t width, int32_t height, int64_t pitch_bytes,
                                            int32_t dtype, void* d_segments, uint32_t capacity, uint32_t* d_count,
                                            void* cuda_stream) {
  if (!d_image || !d_segments || !d_count || width < 1 || height < 1 || (dtype != SBMT_U8 && dtype != SBMT_U16) ||
      pitch_bytes < (int64_t)width * dtype)
    return static_fail(SBMT_EINVAL, "bad arguments");
  // u16 pixels are read with 2-byte loads: an odd pitch or address would be
  // a misaligned access
  if (dtype == SBMT_U16 && ((pitch_bytes & 1) || ((uintptr_t)d_image & 1)))
    return static_fail(SBMT_EINVAL, "a u16 image needs an even pitch and an even address");
  const size_t wpr = ((size_t)width + 1 + 31) / 32, wpc = ((size_t)height + 1 + 31) / 32;
  const size_t need = 4 + wpr * ((size_t)height + 1) + wpc * ((size_t)width + 1);
  if (width > 4096 || height > 4096 || need > kStaticWords)
    return static_fail(SBMT_EINVAL, "image too large for the static working memory (at most 4096 x 4096 pixels)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return static_fail(SBMT_ECUDA, "no current CUDA device");
  unsigned int* base;
  {
    // set-up once per device, with that device current: the device address
    // of the static array (its host-side name is only a stand-in)
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p) return static_fail(SBMT_ECUDA, cudaGetErrorString(e));
      g_static_ptr[dev] = (unsigned int*)p;
    }
    base = g_static_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long* nvtx = (unsigned long long*)base;  // words 0-1
  u32* nseg = base + 2;
  u32* err = base + 3;
  u32* vrow = base + 4;
  u32* vcol = vrow + wpr * ((size_t)height + 1);
  // the array keeps the previous call's contents: clear the counters
  if (cudaMemsetAsync(base, 0, 4 * sizeof(u32), st) != cudaSuccess)
    return static_fail(SBMT_ECUDA, "clearing the counters failed");
  launch_corner_bits((const unsigned char*)d_image, pitch_bytes, dtype, width, height, vrow, (int)wpr, vcol,
                     (int)wpc, nvtx, st);
  launch_segments((const unsigned char*)d_image, pitch_bytes, dtype, width, height, vrow, (int)wpr, vcol, (int)wpc,
                  (Seg*)d_segments, capacity, nseg, err, st);
  // the count, or NONE when the extraction met an inconsistency (a run
  // without an end vertex: never for a valid image)
  k_static_count<<<1, 32, 0, st>>>(nseg, err, d_count);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(SBMT_ECUDA, cudaGetErrorString(e));
  return SBMT_OK;
}
