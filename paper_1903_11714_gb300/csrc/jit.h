// Run-time specialisation of the single-lattice sweep kernel to one lattice's
// acceptance thresholds (jit.cu).
#pragma once
#include <cstdint>
#include <string>

namespace ising {

// The single-lattice instance of the packed sweep kernel (NT = threads, whole rows
// or column blocks) compiled with the thresholds (t2, t4, all2, all4) of one
// lattice as constants, as a kernel handle that cudaLaunchKernel and
// cudaFuncSetAttribute accept.  Built once per distinct argument set and process
// (NVRTC to a cubin for this GPU's architecture, loaded with cudaLibraryLoadData)
// and cached.  Returns nullptr, with the reason in *why, when NVRTC cannot be
// loaded, the compile or load fails, or specialisation is switched off.
const void* jit_sweep_kernel(int threads, bool blocks, uint32_t t2, uint32_t t4, uint32_t all2, uint32_t all4,
                             std::string* why, bool one = true);
// one = false: the multi-lattice instance (descriptors read from the tile table; for a
// batch whose lattices all have these thresholds; blocks: it may hold column blocks).

// The three-dimensional sweep kernel (NT = threads, G words per group) compiled for
// thresholds t[0..2] (h = 2, 4, 6) and their always masks: out[0] the colour-0
// instance (no counts), out[1] the colour-1 instance (fused M/E counts).  One NVRTC
// compile per distinct argument set and process.  false, with *why, as above.
bool jit_cubic_kernels(int threads, int G, const uint32_t t[3], const uint32_t all[3], const void* out[2],
                       std::string* why);

// Process-wide switch (default on); off makes jit_sweep_kernel return nullptr.
void jit_set_enabled(bool on);
bool jit_enabled();

// Milliseconds spent compiling and loading specialised kernels in this process.
double jit_compile_ms();

}  // namespace ising
