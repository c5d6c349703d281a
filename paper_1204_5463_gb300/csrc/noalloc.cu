// dw_apply_f32_noalloc: the FP32 path of dw_apply (convert the input to the
// internal FP32 layout, apply D, convert back) for callers that must not
// allocate device memory -- code running inside a pre-reserved memory pool,
// under an allocator that forbids cudaMalloc, or in a process whose memory
// budget is fixed at start-up. The internal-layout copies of the links and of
// the input/output fields live in one file-scope __device__ array instead of
// buffers of a context.
#include <map>
#include <mutex>

#include "internal.h"

namespace {

// 480 bytes per site (FP32 links 288 + input 96 + output 96) for up to 4096
// sites. Every device that loads the library holds this array until exit.
constexpr long long kNoAllocMaxSites = 4096;
constexpr size_t kNoAllocBytes = 480 * kNoAllocMaxSites;
static __device__ __align__(256) unsigned char g_dw_noalloc_scratch[kNoAllocBytes];

// Host code cannot use g_dw_noalloc_scratch as a device address (it names a
// host-side shadow); the device address is looked up once per device.
std::mutex g_mu;
std::map<int, char*> g_addr;

int scratch_address(char** out) {
    int dev = 0;
    DW_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_addr.find(dev);
    if (it != g_addr.end()) {
        *out = it->second;
        return DW_OK;
    }
    void* p = nullptr;
    DW_CUDA_TRY(cudaGetSymbolAddress(&p, g_dw_noalloc_scratch));
    g_addr[dev] = static_cast<char*>(p);
    *out = static_cast<char*>(p);
    return DW_OK;
}

}  // namespace

using namespace dwk;

extern "C" int dw_apply_f32_noalloc(const int* dims, double m0, const double* U, const double* in, double* out,
                                    void* cuda_stream) {
    if (!dims || !U || !in || !out) return fail(DW_EINVAL, "null argument");
    Geom g{};
    g.V = 1;
    g.B = 1;
    g.ndom = 1;
    // the size check runs on the partial products, so huge extents cannot
    // overflow or wrap to a volume that seems to fit the scratch
    if (!lattice_volume(dims, kNoAllocMaxSites, &g.V))
        return fail(DW_EINVAL,
                    "dw_apply_f32_noalloc needs extents >= 2 and at most 4096 sites (scratch is a fixed device array)");
    for (int j = 0; j < 4; ++j) {
        g.d[j] = g.b[j] = dims[j];
        g.nb[j] = 1;
    }
    char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const long long V = g.V;
    char* links = base;                               // 288 V
    char* fin = base + link_bytes(P32, kNoAllocMaxSites);   // 96 V
    char* fout = fin + spinor_bytes(P32, kNoAllocMaxSites);  // 96 V
    if ((rc = launch_gauge_convert(P32, U, links, V, st))) return rc;
    if ((rc = launch_to_internal(P32, in, fin, V, 1, st))) return rc;
    const long long fb = spinor_bytes(P32, V);
    FieldRef fi{fin, fb, 0, 0}, fo{fout, fb, 0, 0};
    if ((rc = launch_dw(P32, P32, P32, g, m0, fi, fo, links, nullptr, 1, nullptr, st))) return rc;
    if ((rc = launch_from_internal(P32, fout, out, V, 1, st))) return rc;
    DW_CUDA_TRY(cudaStreamSynchronize(st));
    return DW_OK;
}
