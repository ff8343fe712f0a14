// Host build of the library's integer-pipe FP64 helpers (pdg_fp.cuh), for
// tests/test_fp_host.py: the same source the kernels compile, checked against
// IEEE arithmetic done by Python.
#include <stdint.h>

#include "pdg_fp.cuh"

extern "C" void pdg_host_rcp_bits(const uint64_t* w, uint64_t* out, int32_t* ok, int64_t n) {
  for (int64_t i = 0; i < n; i++) {
    bool o;
    out[i] = pdg::rcp_rn_bits(w[i], &o);
    ok[i] = o ? 1 : 0;
  }
}

extern "C" void pdg_host_fixed_bits(const uint64_t* hi, const uint64_t* lo, const int32_t* S, uint64_t* out,
                                    int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = pdg::fixed_hl_to_bits(hi[i], lo[i], S[i]);
}
