// Device and launch helpers of the GNP operator's kernels (paired float32 multiply-adds,
// programmatic dependent launch).
#pragma once

#include "internal.h"

namespace gnp {

// d += a * b on two float32 lanes at once (fma.rn.f32x2: each lane an fmaf).
__device__ __forceinline__ void ffma2(float& dx, float& dy, float ax, float ay, float bx, float by) {
  asm("{\n\t.reg .b64 ta, tb, td;\n\t"
      "mov.b64 ta, {%2, %3};\n\tmov.b64 tb, {%4, %5};\n\tmov.b64 td, {%0, %1};\n\t"
      "fma.rn.f32x2 td, ta, tb, td;\n\tmov.b64 {%0, %1}, td;\n\t}"
      : "+f"(dx), "+f"(dy)
      : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}

// Programmatic dependent launch: each layer is launched while the previous one drains.
// A layer loads its tile's row pointers (the matrix, never written), then waits for the
// previous grid to complete and flush (griddepcontrol.wait) before any read of data a
// previous kernel wrote; it releases its own dependents once its epilogue is done.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialization (the kernel calls pdl_wait before it
// reads anything an earlier kernel wrote).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TILE);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace gnp
