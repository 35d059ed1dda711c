// grouped.cu -- grouped (batched) Scheme I products.
#include "emu_internal.h"
#include "emu_handle.h"

namespace emu {
void grouped_release(emu_handle_s* h) { (void)h; }
}  // namespace emu
