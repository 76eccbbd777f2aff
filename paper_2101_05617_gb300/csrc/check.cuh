// Bounds-checked builds (compiled with -DSW_CHECK; libswepi_check.so).
//
// The kernels that index through the grid tables (the interface lines'
// element and edge numbers) or issue bulk copies from computed ranges test
// those indices before they use them.  A failed test records a code in a
// device word of its translation unit (the first code wins) and the thread
// skips the accesses the index would drive: the kernel neither traps nor
// touches memory out of range, and the host learns of it through
// sw_check_status, which reads and clears every translation unit's word.  In
// the default build every test compiles to nothing.
#pragma once

#include <cuda_runtime.h>

#include "swepi_internal.h"

namespace swepi {

// codes recorded by the checks
enum CheckCode : unsigned {
  CHK_FACE_LINE = 1,     // an interface line's element or edge number out of range (face kernels)
  CHK_TILE_RANGE = 2,    // a staged tile's copy range outside its arrays, or a misaligned bulk copy
  CHK_ENS_TASK = 3,      // an ensemble task's member, element range or vector index out of range
};

#ifdef SW_CHECK
constexpr bool kChecked = true;
// one word per translation unit (static: no relocatable device code needed)
static __device__ unsigned int sw_check_word;
__device__ __forceinline__ void check_fail(unsigned code) { atomicCAS(&sw_check_word, 0u, code); }
// host side: this translation unit's word, cleared after the read (0: no failure)
#define SW_CHECK_READER(name)                                                             \
  unsigned name() {                                                                       \
    unsigned v = 0, z = 0;                                                                \
    if (cudaMemcpyFromSymbol(&v, sw_check_word, sizeof(v)) != cudaSuccess) return ~0u;   \
    if (cudaMemcpyToSymbol(sw_check_word, &z, sizeof(z)) != cudaSuccess) return ~0u;     \
    return v;                                                                             \
  }
#else
constexpr bool kChecked = false;
__device__ __forceinline__ void check_fail(unsigned) {}
#define SW_CHECK_READER(name) \
  unsigned name() { return 0u; }
#endif

// the element and edge numbers of an interface line on a grid of `nodes`
// solution points (NS^2 per element)
template <int NS>
__device__ __forceinline__ bool face_line_ok(const FaceLine& L, long long nodes) {
  if (!kChecked) return true;
  const long long ne = nodes / (NS * NS);
  const bool ok = L.owner >= 0 && L.owner < ne && L.nbr >= 0 && L.nbr < ne && (unsigned)L.owner_edge < 4u &&
                  (unsigned)L.nbr_edge < 4u;
  if (!ok) check_fail(CHK_FACE_LINE);
  return ok;
}

// readers of the translation units with checks (sw_check_status)
unsigned check_word_dfr();
unsigned check_word_split();
unsigned check_word_tile();
unsigned check_word_ensemble();

}  // namespace swepi
