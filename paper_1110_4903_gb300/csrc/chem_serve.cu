// chem_serve.cu -- serving loop (continuous batching); filled in below.
#include "chem_handle.h"

namespace chem {
void destroy_serving(Handle *h) { (void)h; }
}  // namespace chem
