// Which memory a kernel launched for a context on device `ctx_device` may
// touch: device memory of that same device, or managed memory (migrated on
// demand).  Memory of another device is refused: with peer access off, a
// kernel that reads it faults.  Host and unregistered memory are refused by
// the entry points that take device arrays only.  Plain integers so that the
// rule can be checked on a host without a GPU (the values are those of
// cudaMemoryType: 0 unregistered, 1 host, 2 device, 3 managed).
#pragma once

namespace klecgc {

inline bool device_array_usable(int mem_type, int mem_device, int ctx_device) {
    if (mem_type == 3) return true;                       // managed
    return mem_type == 2 && mem_device == ctx_device;     // device, same GPU
}

}  // namespace klecgc
