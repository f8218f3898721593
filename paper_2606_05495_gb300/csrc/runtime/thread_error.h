// thread_error.h -- error text of the calling thread's last context-less C ABI call (returned by
// set_last_error(NULL)).
#pragma once

namespace setrt {
void set_thread_error(const char* msg);
const char* thread_error_text();
}  // namespace setrt
