// noalloc.cu -- nbody_accel_noalloc: the force evaluation of nbody_accel with
// its default options (mixed precision, cells of bodies in Morton order,
// compensated sums) on the 1024-body-block kernel shape, with every scratch
// buffer in one fixed device array, for callers that must not allocate GPU
// memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// framework's memory pool or allocator callback (allocating there can
// re-enter the allocator or deadlock), in a real-time loop that must never
// block on the driver's allocator, or in a process that has handed all free
// device memory to another consumer and accounts for every byte up front.
// nbody_accel grows a cached workspace with cudaMalloc; this entry point
// never does.
//
// The scratch is `g_scratch` below, a file-scope __device__ array of
// kScratchBytes (23.3 MiB).  Every GPU on which the library's module
// is loaded holds its own copy until the process exits.  In host code the name
// g_scratch is only a host-side stand-in for the symbol, not a device address:
// the set-up looks up the real address once per device with
// cudaGetSymbolAddress, with that device current, and the kernels receive that
// pointer.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "nbody_internal.cuh"

namespace {

constexpr int64_t kMaxN = NBODY_NOALLOC_MAX_N;      // 65536 bodies
constexpr int kShape = 1;                           // 1024-body i-blocks, 256-body j-tiles
constexpr int kBlock = 1024;
constexpr size_t kJdupBytes = (size_t)kMaxN * nbk::kJdupFloats * sizeof(float);  // 2 MiB
constexpr size_t kCentreBytes = 8192;               // cell centres and 256-body chunk sums (pack_centre_doubles)
constexpr size_t kWordBytes = 256;                  // error word (when the caller passes none), equal-mass flag
constexpr size_t kPermBytes = (size_t)kMaxN * sizeof(int);                       // Morton permutation
constexpr size_t kOrderBytes = (size_t)kMaxN * 16 + ((size_t)64 << 10);         // radix-sort scratch
constexpr size_t kPartialBytes = (size_t)20 << 20;  // split i-block partial sums
constexpr size_t kOffCentres = kJdupBytes;
constexpr size_t kOffWords = kOffCentres + kCentreBytes;
constexpr size_t kOffPerm = kOffWords + kWordBytes;
constexpr size_t kOffOrder = kOffPerm + kPermBytes;
constexpr size_t kOffPartial = kOffOrder + kOrderBytes;
constexpr size_t kScratchBytes = kOffPartial + kPartialBytes;
static_assert((3 * (kMaxN / kBlock) + 3 * (kMaxN / 256)) * sizeof(double) <= kCentreBytes, "centre area too small");
static_assert(kOffPerm % 256 == 0 && kOffOrder % 256 == 0 && kOffPartial % 256 == 0, "areas stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
struct DeviceScratch {
    bool ready = false;
    int status = NBODY_OK;     // outcome of the set-up, kept for later calls
    unsigned char* base = nullptr;
    int num_sms = 0;
};
std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

// Once per device, with that device current: check it and resolve the device
// address of g_scratch.
int setup(int dev, DeviceScratch** out) {
    if (dev < 0 || dev >= kMaxDevices) return NBODY_ENOTSUP;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch& d = g_dev[dev];
    if (!d.ready) {
        int major = 0, minor = 0, sms = 0;
        d.status = NBODY_OK;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            d.status = NBODY_ECUDA;
        } else if (!(major == 10 && minor == 3)) {
            d.status = NBODY_ENOTSUP;
        } else {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || p == nullptr) {
                (void)cudaGetLastError();
                d.status = NBODY_ECUDA;
            } else {
                d.base = static_cast<unsigned char*>(p);
                d.num_sms = sms;
            }
        }
        d.ready = true;
    }
    *out = &d;
    return d.status;
}

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int nbody_accel_noalloc(int64_t n, const double* pos, const float* mass, double eps, float* acc,
                                   float* pot, int* status, void* stream) {
    NB_RANGE("nbody_accel_noalloc");
    if (n < 0 || n > kMaxN || !isfinite(eps) || eps < 0.0) return NBODY_EINVAL;
    if (n > 0 && (pos == nullptr || mass == nullptr || acc == nullptr)) return NBODY_EINVAL;
    if (n == 0) return NBODY_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return NBODY_ECUDA;
    }
    DeviceScratch* d = nullptr;
    const int rc = setup(dev, &d);
    if (rc != NBODY_OK) return rc;
    if (!device_ptr(pos) || !device_ptr(mass) || !device_ptr(acc) || (pot && !device_ptr(pot)) ||
        (status && !device_ptr(status)))
        return NBODY_EINVAL;  // host arrays would need staging buffers, i.e. allocation

    const int64_t npad = (n + kBlock - 1) / kBlock * kBlock;
    const size_t need = nbk::force_partial_doubles_for(kShape, pot != nullptr, true, true, npad, d->num_sms) *
                        sizeof(double);
    // a device with more SMs than the partial-sum area was sized for
    if (need > kPartialBytes || nbk::order_scratch_bytes(n) > kOrderBytes) return NBODY_ENOMEM;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = d->base;
    float* jdup = reinterpret_cast<float*>(base);
    double* centres = reinterpret_cast<double*>(base + kOffCentres);
    int* word = status ? status : reinterpret_cast<int*>(base + kOffWords);
    int* uni = reinterpret_cast<int*>(base + kOffWords + 128);
    int* perm = reinterpret_cast<int*>(base + kOffPerm);
    void* order_scratch = base + kOffOrder;
    double* partial = reinterpret_cast<double*>(base + kOffPartial);

    // The same sequence nbody_accel queues for these options.  Only the error
    // word must start at zero: the sort, the equal-mass check and the pack
    // kernel write everything they later read, and each partial slot is
    // written before the fixup reads it.
    bool ok = cudaMemsetAsync(word, 0, sizeof(int), st) == cudaSuccess;
    ok = ok && nbk::spatial_order(n, pos, perm, order_scratch, st) == cudaSuccess;
    ok = ok && nbk::uniform_mass_flag(n, mass, uni, st) == cudaSuccess;
    ok = ok && nbk::pack_f64(n, npad, kBlock, const_cast<double*>(pos), nullptr, nullptr, mass, 0.0, 0.0, false,
                             jdup, centres, st, perm, word) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        return NBODY_ECUDA;
    }
    nbk::ForceArgs a;
    a.jdup = jdup;
    a.centres = centres;
    a.eps2 = (float)(eps * eps);
    a.n = n;
    a.npad = npad;
    a.perm = perm;
    a.acc = acc;
    a.pot = pot;
    a.partial = partial;
    a.err = word;
    a.summation = 1;
    a.uni = uni;
    int launched = 0;
    if (nbk::force_launch(kShape, a, d->num_sms, st, &launched) != cudaSuccess) {
        (void)cudaGetLastError();
        return NBODY_ECUDA;
    }
    return NBODY_OK;
}
