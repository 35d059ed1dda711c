// extras.cu -- release of optional handle state (grouped plans, selector,
// host-buffer staging, trace).
#include "emu_handle.h"

namespace emu {
void grouped_release(emu_handle_s* h);
void selector_release(emu_handle_s* h);
void hostio_release(emu_handle_s* h);
void handle_release_extras(emu_handle_s* h) {
  grouped_release(h);
  selector_release(h);
  hostio_release(h);
  trace_release(h);
}
}  // namespace emu
