// api.cu -- error state and version of the MSG-MIMC C ABI.
#include <string>

#include "common.cuh"

namespace msg {
namespace {
thread_local std::string g_last_error;
}
void set_error(const std::string& what) { g_last_error = what; }
void clear_error() { g_last_error.clear(); }
}  // namespace msg

extern "C" const char* msg_last_error(void) { return msg::g_last_error.c_str(); }
extern "C" const char* msg_version(void) { return "msg-mimc-gb300 0.1 (sm_103a)"; }
