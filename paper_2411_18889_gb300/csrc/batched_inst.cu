// batched_inst.cu -- one instantiation of the persistent batched kernel
// (batched_kernel.cuh): shape NBK_BSHAPE of kBShapes, with (NBK_BPOT = 1) or
// without the potential.  The library's build compiles this file once per
// (shape, potential) pair, so the kernels compile in parallel.
#include "batched_kernel.cuh"

#if !defined(NBK_BSHAPE) || !defined(NBK_BPOT)
#error "batched_inst.cu is compiled with -DNBK_BSHAPE=<0..5> -DNBK_BPOT=<0|1>"
#endif

#define NBK_CAT3_(a, b, c) a##b##c
#define NBK_CAT3(a, b, c) NBK_CAT3_(a, b, c)

namespace nbk {
namespace {
constexpr BShapeDef kDef = kBShapes[NBK_BSHAPE];
}

BFn NBK_CAT3(batched_fn_, NBK_BSHAPE, NBK_BPOT)() {
    return batched_kernel<kDef.threads, kDef.ibodies, NBK_BPOT != 0, kDef.unroll, kDef.jblock>;
}
}  // namespace nbk
