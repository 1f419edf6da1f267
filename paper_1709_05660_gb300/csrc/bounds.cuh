// Index checks of the bounds-check build (compiled with -DFSI_BOUNDS_CHECK;
// without it every check is the constant true and costs nothing).
//
// A check FSI_IN(i, n, site) is true when 0 <= i < n.  When it fails, the
// first failing site of the translation unit is recorded in a device word
// (a site is FSI_SITE: translation-unit id * 100000 + source line) and the
// caller skips the access; nothing traps.  The host reads and clears the
// words after every compute call (fsi_bounds_site) and turns a recorded site
// into FSI_E_CUDA with the site in the message.
#pragma once

#include <cstdint>

#ifdef FSI_BOUNDS_CHECK
namespace fsi {
namespace bounds {
static __device__ int g_site;   // one per translation unit (no relocatable device code)
}  // namespace bounds
}  // namespace fsi
#define FSI_SITE(tu) ((tu) * 100000 + __LINE__)
#define FSI_IN(i, n, site)                                                              \
  (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n))           \
       ? true                                                                           \
       : (atomicCAS(&fsi::bounds::g_site, 0, (site)), false))
// host reader of this translation unit's word: returns the recorded site and clears it
#define FSI_BOUNDS_READER(name)                                                         \
  int name() {                                                                          \
    int v = 0, z = 0;                                                                   \
    cudaMemcpyFromSymbol(&v, fsi::bounds::g_site, sizeof(int));                         \
    if (v) cudaMemcpyToSymbol(fsi::bounds::g_site, &z, sizeof(int));                    \
    return v;                                                                           \
  }
#else
#define FSI_SITE(tu) 0
#define FSI_IN(i, n, site) true
#define FSI_BOUNDS_READER(name) \
  int name() { return 0; }
#endif
