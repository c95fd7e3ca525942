// Internal helpers shared by the library's translation units (not part of
// the C-ABI): they set the calling thread's sw_last_error().
#pragma once

#include <cstdint>

int32_t sw_internal_fail(int32_t code);  // records code as the last error and returns it
int32_t sw_internal_ok();                // records SW_OK and returns it
