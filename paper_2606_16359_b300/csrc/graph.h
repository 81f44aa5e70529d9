// The captured-graph handle behind fe_graph (include/fenc.h): a CUDA graph of
// a sequence of library launches over fixed device buffers, with the buffers
// that fe_graph_launch_host copies in and out.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

struct fe_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    // the captured sequence's external inputs (layer inputs no earlier layer writes)
    // and final outputs (layer outputs no later layer reads), in layer order
    struct Io {
        void* dev;
        size_t bytes;
    };
    std::vector<Io> in, out;
    std::vector<uint32_t> out_level;  // level of each final output ciphertext array
    uint32_t host_out_level = UINT32_MAX;  // outputs copied to the host at this level (UINT32_MAX: their own)
    size_t N = 0;
};
