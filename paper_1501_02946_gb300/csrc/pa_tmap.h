// pa_tmap.h -- host-side encoding of TMA tensor maps (cuTensorMapEncodeTiled,
// reached through the runtime's driver entry-point query, so the library
// needs no link against the driver library) for the tile copies of the
// pipelined kernels.  Every map describes float32 data; boxes are at most
// 256 elements per dimension; base addresses and row pitches 16-byte aligned.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

namespace pa {

// The driver's encoder, looked up once (null if unavailable).
static inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

// 2-D float map: rows of `inner` floats, `outer` rows, row pitch in bytes;
// box bx x by.  False (map zeroed) when unavailable.
static inline bool encode_2d(const void *base, uint64_t inner, uint64_t outer, uint64_t pitch, uint32_t bx, uint32_t by,
                      CUtensorMap *map) {
  std::memset(map, 0, sizeof(*map));
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode || (reinterpret_cast<uintptr_t>(base) & 15u) || (pitch & 15u) || bx > 256 || by > 256) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {pitch};
  const cuuint32_t box[2] = {bx, by};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    std::memset(map, 0, sizeof(*map));
    return false;
  }
  return true;
}

// 3-D float map: dims d0 (contiguous), d1, d2 with byte pitches p1, p2; box b0 x b1 x b2.
static inline int encode_3d(const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t p1, uint64_t p2, uint32_t b0,
                     uint32_t b1, uint32_t b2, CUtensorMap *map) {
  std::memset(map, 0, sizeof(*map));
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode || (reinterpret_cast<uintptr_t>(base) & 15u) || (p1 & 15u) || (p2 & 15u) || b0 > 256 || b1 > 256 ||
      b2 > 256)
    return 0;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {p1, p2};
  const cuuint32_t box[3] = {b0, b1, b2};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    std::memset(map, 0, sizeof(*map));
    return 0;
  }
  return 1;
}

}  // namespace pa
