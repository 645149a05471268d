// graph.h -- the device-driven MAP solve (graph.cu).
#pragma once
#include <vector>

#include "ctx.h"

namespace plc {

// One solve as one CUDA graph launch (same iteration as newton_map).
template <typename TC>
plc_status newton_map_graph(plc_ctx* c, const int32_t* N, const double* w, double nbar,
                            double* s_out, const plc_opts& o, plc_stats* st);

// The cached graph of a batch of contexts.
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;
  std::vector<double> key_val;
  ~BatchGraph();
};

plc_status batch_map(BatchGraph* b, const std::vector<plc_ctx*>& cs, const int32_t* const* N,
                     const double* const* w, const double* nbar, double* const* s,
                     const plc_opts& o, plc_stats* stats, cudaStream_t stream);

void graph_release(plc_ctx* c);

}  // namespace plc
