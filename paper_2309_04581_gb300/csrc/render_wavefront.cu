// Wavefront engine (not built yet): the megakernel is the only engine.
#include <cuda_runtime.h>

#include "common.h"

namespace mrf {

bool wavefront_available() { return false; }
size_t wavefront_scratch_bytes(const RenderParams &) { return 0; }
cudaError_t launch_render_wavefront(const RenderParams &, void *, size_t, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace mrf
