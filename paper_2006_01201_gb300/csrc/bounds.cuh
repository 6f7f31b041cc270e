// bounds.cuh -- internal: index checks of the debug build of the library.
//
// Compiled with -DPANO_BOUNDS_CHECK (the `check` variant of build.build()),
// PANO_AT(base, off, n, site) checks that `off` lies in [0, n), the n
// elements of the array that starts at `base`, before the access. A
// violation is counted and the first one (site, offset, bound) recorded in a
// device word of the including translation unit; the offset is then clamped
// into range, so the access itself stays in bounds and nothing traps. The
// host reads and clears the record with PANO_BOUNDS_READER. In the normal
// build PANO_AT(base, off, n, site) is base[off] and no record exists.
#pragma once

#include <cuda_runtime.h>

#ifdef PANO_BOUNDS_CHECK
namespace {
__device__ unsigned g_pano_oob[4];  // count, site, offset, bound of the first violation
}  // namespace

namespace pano {
template <class T>
__device__ __forceinline__ T* checked_at(T* base, long long off, long long n, int site) {
    if (off < 0 || off >= n) {
        if (atomicAdd(&g_pano_oob[0], 1u) == 0u) {
            g_pano_oob[1] = (unsigned)site;
            g_pano_oob[2] = (unsigned)off;
            g_pano_oob[3] = (unsigned)n;
        }
        off = off < 0 ? 0 : n - 1;
    }
    return base + off;
}
// an index i into [0, n): an image column or row before its address is formed
__device__ __forceinline__ int checked_idx(int i, int n, int site) {
    if (i < 0 || i >= n) {
        if (atomicAdd(&g_pano_oob[0], 1u) == 0u) {
            g_pano_oob[1] = (unsigned)site;
            g_pano_oob[2] = (unsigned)i;
            g_pano_oob[3] = (unsigned)n;
        }
        i = i < 0 ? 0 : n - 1;
    }
    return i;
}
// `width` consecutive elements from `off` (a vector access): a clamped
// offset is rounded down to a multiple of `width`, so it keeps the
// alignment that every valid offset of such an access has.
template <class T>
__device__ __forceinline__ T* checked_vec(T* base, long long off, int width, long long n, int site) {
    if (off < 0 || off + width > n) {
        if (atomicAdd(&g_pano_oob[0], 1u) == 0u) {
            g_pano_oob[1] = (unsigned)site;
            g_pano_oob[2] = (unsigned)off;
            g_pano_oob[3] = (unsigned)n;
        }
        off = off < 0 ? 0 : (n - width) / width * width;
    }
    return base + off;
}
}  // namespace pano
#define PANO_AT(base, off, n, site) (*pano::checked_at((base), (long long)(off), (long long)(n), (site)))
// an index i into [0, n) (an image column or row before its address is formed)
#define PANO_IDX(i, n, site) pano::checked_idx((i), (n), (site))
// a condition that valid inputs never meet (an iteration limit reached):
// recorded like an index outside its array, with offset and bound 0
#define PANO_FLAG(cond, site) ((cond) ? (void)pano::checked_idx(0, 0, (site)) : (void)0)
// a vector of `width` elements of base's type starting at `off`
#define PANO_VEC(VT, base, off, width, n, site) \
    (*reinterpret_cast<VT*>(pano::checked_vec((base), (long long)(off), (width), (long long)(n), (site))))
// host: add this unit's record to out[4] (count summed, first site kept) and clear it
#define PANO_BOUNDS_READER(fn)                                                   \
    cudaError_t fn(unsigned* out) {                                              \
        unsigned r[4] = {0, 0, 0, 0};                                            \
        cudaError_t e = cudaMemcpyFromSymbol(r, g_pano_oob, sizeof(r));          \
        if (e != cudaSuccess) return e;                                          \
        if (r[0] && !out[0]) { out[1] = r[1]; out[2] = r[2]; out[3] = r[3]; }    \
        out[0] += r[0];                                                          \
        const unsigned z[4] = {0, 0, 0, 0};                                      \
        return cudaMemcpyToSymbol(g_pano_oob, z, sizeof(z));                     \
    }
#else
#define PANO_AT(base, off, n, site) ((base)[off])
#define PANO_IDX(i, n, site) (i)
#define PANO_FLAG(cond, site) ((void)sizeof(cond))
#define PANO_VEC(VT, base, off, width, n, site) (*reinterpret_cast<VT*>((base) + (off)))
#define PANO_BOUNDS_READER(fn) \
    cudaError_t fn(unsigned*) { return cudaSuccess; }
#endif
