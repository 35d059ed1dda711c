// select.cu -- learned slice-count selector.
#include "emu_internal.h"
#include "emu_handle.h"

namespace emu {
void selector_release(emu_handle_s* h) { (void)h; }
}  // namespace emu
