// host_path.h -- host-buffer entry points (host_path.cu): the pipelined
// copies of keccak_batch_uniform_host and page-locked host memory placed near
// the GPU.
#pragma once

namespace kb {

// Frees the pipeline buffers and streams, and forgets the host-path
// decisions, of device `device`.
void release_host_pipeline(int device);

}  // namespace kb
