// Host-side declarations of the CSR build.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <algorithm>

namespace kc {

struct CsrLayout {
  size_t status, keys0, keys1, hist, offs, total;
  long long N;      // keys = 2 * edges
  long long chunk;  // keys per CTA (multiple of the 4096-key tile)
  int grid;
  int B;            // bits per vertex id
};

CsrLayout csr_layout(long long n, long long E, int sms);
cudaError_t csr_build_launch(const CsrLayout& L, char* ws, long long n, long long E, const int* src,
                             const int* dst, long long* off_out, int* adj_out, long long* m_out,
                             cudaStream_t stream);

}  // namespace kc
