// Test probe: the library's host-side sparse approximate inverse
// (paper_2003_11679_gb300/csrc/spai.cpp) behind one C function, compiled
// together with that file by tests/test_spai_host.py for a CPU check.
#include <complex>
#include <string>
#include <vector>

#include "../paper_2003_11679_gb300/csrc/internal.h"

namespace sie {
int64_t spai_host(const CsrPattern& P, const std::complex<double>* val, std::complex<double>* M);
void set_error(const std::string&) {}
}  // namespace sie

extern "C" long long spai_probe(long long n, const long long* rp, const int* col, const double* val, double* M)
{
    sie::CsrPattern P;
    P.row_ptr.assign(rp, rp + n + 1);
    P.col.assign(col, col + rp[n]);
    return sie::spai_host(P, reinterpret_cast<const std::complex<double>*>(val),
                          reinterpret_cast<std::complex<double>*>(M));
}
