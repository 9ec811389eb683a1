// Host-side helpers shared by the libgnnmp translation units: error state.
#pragma once

#include <cstdarg>
#include <cstdio>
#include <string>

#include "gnnmp.h"

namespace gnn {

// Records `code` with a printf-style message as this thread's last error and returns it.
int set_error(int code, const char* fmt, ...);
void clear_error();

}  // namespace gnn

#define GNN_REQUIRE(cond, code, ...)                        \
    do {                                                    \
        if (!(cond)) return ::gnn::set_error((code), __VA_ARGS__); \
    } while (0)
