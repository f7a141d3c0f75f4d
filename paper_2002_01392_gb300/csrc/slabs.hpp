// Slab plan of fc_deriv_z_host (host only; also compiled into the host-check
// library so that CPU tests can check it): which y rows of which field each
// staged slab moves.
#pragma once
#include <algorithm>
#include <cstddef>
#include <vector>

namespace fcns {

struct Slab {
  int b;              // field
  long long y0, yc;   // first y row and row count
};

// Slabs of y rows (all z and x of a field) of at most about slab_bytes of
// input (yrow = bytes of one y row over all z), an even number of rows each
// (so that the kernel pairs the same lines as a call on the whole field; only
// a field's last slab may be odd, when Ny is), the slabs of a field as equal
// as that allows; the first slab of the call about a quarter of the others, so
// that the device-to-host copies start sooner.  Returns the staging rows per
// slot (every slab has at most that many rows).
inline long long plan_slabs(int batch, long long Ny, size_t yrow, size_t slab_bytes, std::vector<Slab>* out) {
  out->clear();
  long long Yc = (long long)std::max<size_t>(2, slab_bytes / yrow);
  Yc -= Yc % 2;
  if (Yc >= Ny) {
    Yc = Ny;
  } else {
    const long long ns = (Ny + Yc - 1) / Yc;
    Yc = (Ny + ns - 1) / ns;
    Yc += Yc % 2;
  }
  for (int b = 0; b < batch; ++b) {
    long long y0 = 0;
    if (b == 0 && Yc < Ny) {
      long long first = std::max<long long>(2, Yc / 4);
      first -= first % 2;
      out->push_back({0, 0, first});
      y0 = first;
    }
    const long long rest = Ny - y0, ns = (rest + Yc - 1) / Yc;
    long long each = ns > 0 ? (rest + ns - 1) / ns : 0;
    each += each % 2;
    if (each > Yc) each = Yc;
    for (; y0 < Ny; y0 += each) out->push_back({b, y0, std::min<long long>(each, Ny - y0)});
  }
  return Yc;
}

}  // namespace fcns
