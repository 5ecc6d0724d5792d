// Allocation-free variant of nefe_cell_bin for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's memory
// pool or allocator and must not create allocations of its own, real-time loops that must
// never enter the driver's allocator, or processes whose device memory is fully reserved up
// front.  nefe_cell_bin_noalloc does the same work as nefe_cell_bin but keeps its scratch
// (descriptors, mirror coordinates, unwrapped cell indices, occupancy counts and cursors) in
// one file-scope __device__ array of fixed size, so it calls no cudaMalloc / cudaFree /
// cudaMallocAsync and no allocating library routine.
#include <cstring>
#include <mutex>

#include "nefe.h"
#include "nefe_dev.h"
#include "nefe_host.h"
#include "nefe_launch.h"

namespace nefe {
namespace {

// Scratch layout (bytes), in order: DevSys | DevState | tile table | xs | xa | q | counts |
// cursors.  The mirror arrays use float4 (the entry point runs the FP32 cell kernels).
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffSys = 0;
constexpr size_t kOffSt = align_up(kOffSys + sizeof(DevSys));
constexpr size_t kOffTile = align_up(kOffSt + sizeof(DevState));
constexpr size_t kOffXs = align_up(kOffTile + sizeof(int) * (NEFE_NOALLOC_MAX_ATOMS / kTile + 1));
constexpr size_t kOffXa = align_up(kOffXs + sizeof(float4) * NEFE_NOALLOC_MAX_ATOMS);
constexpr size_t kOffQ = align_up(kOffXa + sizeof(float4) * NEFE_NOALLOC_MAX_ATOMS);
constexpr size_t kOffCount = align_up(kOffQ + sizeof(int4) * NEFE_NOALLOC_MAX_ATOMS);
constexpr size_t kOffCursor = align_up(kOffCount + sizeof(int) * NEFE_NOALLOC_MAX_CELLS);
constexpr size_t kScratchBytes = align_up(kOffCursor + sizeof(int) * NEFE_NOALLOC_MAX_CELLS);

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(void** out) {
    int dev = 0;
    NEFE_CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NEFE_EINVAL, "device index %d above %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return NEFE_OK;
}

// Writes the one-system descriptors (passed by value, so the call issues no host-to-device
// copy from host memory), the tile table (every tile belongs to system 0) and zeroed
// occupancy counts into the scratch.
__global__ void k_noalloc_init(DevSys hs, DevState st, DevSys* dsys, DevState* dst, int* tile_sys, int ntiles,
                               int* counts, int ncells) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (t == 0) {
        *dsys = hs;
        *dst = st;
    }
    for (int i = t; i < ntiles; i += stride) tile_sys[i] = 0;
    for (int i = t; i < ncells; i += stride) counts[i] = 0;
}

}  // namespace
}  // namespace nefe

using namespace nefe;

extern "C" int nefe_cell_bin_noalloc(const double* x, int n, const double box[3], double rcs,
                                     int ncell3[3], int* cell_of, int* cell_start, int* perm,
                                     int ncell_cap, void* stream) {
    if (n < 0 || !box || !ncell3 || (n > 0 && (!x || !cell_of || !perm)) || !cell_start)
        return fail(NEFE_EINVAL, "nefe_cell_bin_noalloc: bad argument");
    if (n > NEFE_NOALLOC_MAX_ATOMS)
        return fail(NEFE_EINVAL, "nefe_cell_bin_noalloc: n = %d above the fixed maximum of %d atoms", n,
                    NEFE_NOALLOC_MAX_ATOMS);
    int rc = check_box(box, rcs);
    if (rc) return rc;
    int n3[3];
    if (!host_grid(box, rcs, n3)) return fail(NEFE_EINVAL, "nefe_cell_bin_noalloc: fewer than 2 cells on an axis");
    const long long total = (long long)n3[0] * n3[1] * n3[2];
    if (total > NEFE_NOALLOC_MAX_CELLS)
        return fail(NEFE_EINVAL, "nefe_cell_bin_noalloc: %lld cells above the fixed maximum of %d", total,
                    NEFE_NOALLOC_MAX_CELLS);
    if (total > ncell_cap) return fail(NEFE_EINVAL, "nefe_cell_bin_noalloc: %lld cells above capacity %d", total, ncell_cap);
    for (int k = 0; k < 3; ++k) ncell3[k] = n3[k];
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        NEFE_CU(cudaMemsetAsync(cell_start, 0, sizeof(int) * (size_t)(total + 1), s));
        return NEFE_OK;
    }
    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char* p = static_cast<unsigned char*>(base);
    const int ntiles = (n + kTile - 1) / kTile;

    DevSys hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.off = 0; hs.n = n; hs.tile0 = 0; hs.ntile = ntiles; hs.cell0 = 0; hs.ncell_cap = (int)total;
    hs.rcs = rcs; hs.pair = -1; hs.mass_e = 1.0;
    DevState st;
    std::memset(&st, 0, sizeof(st));
    for (int k = 0; k < 3; ++k) st.box[k] = box[k];
    st.rebuild = 1;
    // descriptors, tile table and zeroed occupancy counts, all written by one kernel
    {
        const int work = ntiles > (int)total ? ntiles : (int)total;
        const int blocks = (work + 255) / 256 < 152 ? (work + 255) / 256 : 152;
        k_noalloc_init<<<blocks, 256, 0, s>>>(hs, st, reinterpret_cast<DevSys*>(p + kOffSys),
                                               reinterpret_cast<DevState*>(p + kOffSt),
                                               reinterpret_cast<int*>(p + kOffTile), ntiles,
                                               reinterpret_cast<int*>(p + kOffCount), (int)total);
        NEFE_CU(cudaGetLastError());
    }

    Bufs b;
    std::memset(&b, 0, sizeof(b));
    b.sys = reinterpret_cast<DevSys*>(p + kOffSys);
    b.st = reinterpret_cast<DevState*>(p + kOffSt);
    b.tile_sys = reinterpret_cast<int*>(p + kOffTile);
    b.x = const_cast<double*>(x);
    b.xs = p + kOffXs;
    b.xa = p + kOffXa;
    b.q = reinterpret_cast<int4*>(p + kOffQ);
    b.cell_count = reinterpret_cast<int*>(p + kOffCount);
    b.cell_cursor = reinterpret_cast<int*>(p + kOffCursor);
    b.cell_of = cell_of;
    b.perm = perm;
    b.cell_start = cell_start;
    b.ntot = n;
    launch_cells(b, NEFE_FP32, ntiles, 1, 1, s, nullptr);
    NEFE_CU(cudaGetLastError());
    return NEFE_OK;
}
