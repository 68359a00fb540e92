// Width measurement that allocates nothing (rsos_width_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// width: code that runs under a fixed memory budget handed out once at start
// (an arena owned by another framework), real-time loops in which an
// allocation would synchronise the device, or jobs whose caller-owned buffer
// was sized for the lattice alone.  For them this entry point measures a
// multisurface lattice given by plain device pointers, using as scratch a
// file-scope device array that every GPU loading the library holds until the
// process exits.  It runs the same measurement kernels as rsos_width.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rsos.h"
#include "rsos_launch.h"

namespace {

// Scratch of the measurement: rel(x, 0) per surface, per-column-block sums,
// and the 128-bit per-surface totals.  Every call overwrites what it reads:
// nothing has to start at zero.
constexpr size_t kScratchBytes = (size_t)RSOS_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RSOS_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return RSOS_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RSOS_OK;
}

}  // namespace

extern "C" int rsos_width_noalloc(const rsos_params* params, const uint32_t* planes, const int64_t* h00,
                                  int64_t* sums, void* stream)
{
    if (!params || !planes || !h00 || !sums) return RSOS_EINVAL;
    size_t job_bytes = 0;
    int rc = rsos_required_bytes(params, &job_bytes);
    if (rc) return rc;
    if (params->surfaces < 2) return RSOS_EINVAL;  // the plain path keeps absolute heights
    const int T = params->tile_x == 0 ? 8 : params->tile_x;
    rsos::JobDev J{};
    J.planes = const_cast<uint32_t*>(planes);
    J.h00 = const_cast<int64_t*>(h00);
    J.L = params->L;
    J.T = T;
    J.nT = params->tiling == 1 ? rsos::gen_classes(params->L, T) : params->L / T;  // class columns per row
    J.NW = (params->surfaces + 31) / 32;
    J.NWP = J.NW;
    J.N = params->N;
    J.B = rsos::bits_for_step(params->N);
    const int S_pad = J.NW * 32;
    const int ncb = rsos::measure_blocks(J, false);
    const size_t row0_bytes = up256((size_t)S_pad * J.L * 4);
    const size_t partial_bytes = up256((size_t)ncb * S_pad * 2 * 8);
    const size_t rec_bytes = up256((size_t)S_pad * 4 * 8);
    if (row0_bytes + partial_bytes + rec_bytes > kScratchBytes) return RSOS_ERANGE;
    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char* p = static_cast<unsigned char*>(base);
    int32_t* row0 = reinterpret_cast<int32_t*>(p);
    int64_t* partial = reinterpret_cast<int64_t*>(p + row0_bytes);
    int64_t* rec = reinterpret_cast<int64_t*>(p + row0_bytes + partial_bytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = rsos::launch_measure(J, false, S_pad, row0, partial, ncb, rec, 4, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums, rec, (size_t)params->surfaces * 4 * 8, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return RSOS_ECUDA;
    }
    return RSOS_OK;
}
