// TMA tensor-map helpers shared by the kernels that read planes or rows as
// multi-dimensional boxes: the host-side encoder (the CUDA driver API's
// cuTensorMapEncodeTiled, found through the runtime) and the box loads.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <stdint.h>

namespace di {

// cuTensorMapEncodeTiled of the installed driver, or NULL if it has none.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace tc {

// Tiled load of the box at coordinates (c0 innermost, ...) of the tensor map
// into shared memory, completing its bytes on `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

}  // namespace tc
}  // namespace di
