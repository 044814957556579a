// Mixed-precision (tensor-core) sweep: declarations shared with the C ABI.
#pragma once

#include "zbus_internal.cuh"
