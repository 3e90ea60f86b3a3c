// Host-side declarations of the CSR build.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <algorithm>

namespace kc {

struct CsrLayout {
  size_t status, keys0, keys1, hist, offs, rowtot, starts, total;
  long long N;      // keys = 2 * edges
  long long chunk;  // keys per CTA (multiple of the 2,048-key tile), for 2 * edges keys
  long long chunk1; // the same for edges keys (a single graph's build)
  int grid;
  int B;            // bits of the target (local) id in a key
  int Bs;           // bits of the source (global) id in a key
};

// max_graph_n > 0: batched build (targets are graph-local ids below max_graph_n)
CsrLayout csr_layout(long long n, long long E, int sms, long long max_graph_n = 0);
cudaError_t csr_build_launch(const CsrLayout& L, char* ws, long long n, long long E, const int* src,
                             const int* dst, const long long* gv, const long long* eoff, long long G,
                             long long* off_out, int* adj_out, long long* m_out, cudaStream_t stream);

}  // namespace kc
