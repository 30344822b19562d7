// Density filter without any allocation (see topo_filter_noalloc in topo.h).
//
// Some callers cannot allocate GPU memory at the point where they need the
// filter: a framework whose caching allocator already owns the device
// memory, or a loop that must not stall, since cudaMalloc and cudaFree can
// synchronise the whole device.  For them this file keeps the filter's
// scratch in one statically sized device array that every GPU loading the
// library holds until the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"

namespace topo {

namespace {

constexpr long long kNoAllocMaxElems = 1LL << 20;   // largest grid: 1,048,576 elements
constexpr int kNoAllocMaxOffsets = 1024;             // radius <= 6 needs at most 905 offsets
constexpr int kNoAllocMaxDevices = 64;

// layout in doubles: weight sums S [max elems] | g / S [max elems] |
// weights [max offsets] | offsets as int4 (two doubles each) [max offsets]
constexpr long long kScratchDoubles = 2 * kNoAllocMaxElems + 3LL * kNoAllocMaxOffsets;
__device__ __align__(256) double g_filter_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kNoAllocMaxDevices] = {};

// device address of the scratch array for the current device; looked up
// once per device with that device current
topo_status scratch_for_current_device(double** out, std::string* err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        *err = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
        return TOPO_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_filter_scratch);
        if (e != cudaSuccess || !p) {
            *err = std::string("cudaGetSymbolAddress of the filter scratch failed: ") + cudaGetErrorString(e);
            return TOPO_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return TOPO_OK;
}

// Neighbour table of radius r written on the device by one thread, in the
// (dz, dy, dx) order of the host count below: offsets with weight
// w = r - |d| > 0.  |d|^2 is an integer, so the correctly rounded square root
// and the comparison give the same table on host and device.
__global__ void k_filter_table(double r, int R, int4* __restrict__ offs, double* __restrict__ wts) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int n = 0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const double w = r - sqrt((double)(dx * dx + dy * dy + dz * dz));
                if (w > 0.0 && n < kNoAllocMaxOffsets) {
                    offs[n] = make_int4(dx, dy, dz, 0);
                    wts[n] = w;
                    ++n;
                }
            }
}

}  // namespace

}  // namespace topo

using namespace topo;

extern "C" topo_status topo_filter_noalloc(int nx, int ny, int nz, double r, const double* in_dev,
                                           double* out_dev, int transpose, void* stream) {
    std::string err;
    auto fail = [&](topo_status st, const std::string& msg) {
        set_global_error(msg);
        return st;
    };
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(TOPO_BADARG, "grid dimensions must be positive");
    const long long ne = (long long)nx * ny * nz;
    if (ne > kNoAllocMaxElems)
        return fail(TOPO_BADARG, "grid has " + std::to_string(ne) +
                                     " elements; the no-allocation filter supports at most " +
                                     std::to_string(kNoAllocMaxElems));
    if (!(r > 0.0) || r > 6.0) return fail(TOPO_BADARG, "filter radius must be in (0, 6]");
    if (!in_dev || !out_dev || in_dev == out_dev) return fail(TOPO_BADARG, "bad pointers");
    double* scratch = nullptr;
    topo_status st = scratch_for_current_device(&scratch, &err);
    if (st != TOPO_OK) return fail(st, err);
    double* S = scratch;
    double* gs = scratch + kNoAllocMaxElems;
    double* wts = scratch + 2 * kNoAllocMaxElems;
    int4* offs = reinterpret_cast<int4*>(scratch + 2 * kNoAllocMaxElems + kNoAllocMaxOffsets);

    // the neighbour table is written on the device (k_filter_table); the
    // host only counts its entries, so no host memory is copied and the
    // launches depend on the arguments alone
    int n = 0;
    const int R = (int)std::ceil(r);
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx)
                if (r - std::sqrt((double)(dx * dx + dy * dy + dz * dz)) > 0.0 && n < kNoAllocMaxOffsets) ++n;
    cudaStream_t s = (cudaStream_t)stream;
    k_filter_table<<<1, 32, 0, s>>>(r, R, offs, wts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TOPO_CUDA, std::string("filter table launch: ") + cudaGetErrorString(e));

    long long launches = 0;
    const Ctx c{s, &launches};
    Geom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.ne = ne;
    g.nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    if (transpose) {
        // every scratch element read below is written first: nothing needs clearing
        filter_launch(c, g, offs, wts, n, nullptr, S, 2, nullptr);
        divide(c, ne, in_dev, S, gs);
        filter_launch(c, g, offs, wts, n, gs, out_dev, 1, nullptr);
    } else {
        filter_launch(c, g, offs, wts, n, in_dev, out_dev, 0, nullptr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TOPO_CUDA, std::string("filter launch: ") + cudaGetErrorString(e));
    return TOPO_OK;
}
