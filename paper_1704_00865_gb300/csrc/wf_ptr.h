// wf_ptr.h -- where a caller's array lives, decided from what the CUDA
// runtime reports about the pointer.  The rule is kept free of CUDA calls so
// that it can be checked on a host without a GPU.
#pragma once

namespace wf {

enum PtrWhere : int {
  PTR_HOST = 0,          // host memory (pageable or pinned): staged by copies
  PTR_DEVICE = 1,        // memory the current device's kernels may use
  PTR_OTHER_DEVICE = 2   // another GPU's memory: rejected (WF_EINVAL)
};

// query_ok: cudaPointerGetAttributes succeeded; type: its cudaMemoryType
// (0 unregistered, 1 host, 2 device, 3 managed); ptr_dev: its device;
// cur_dev: the current device.  Device memory of another GPU is not taken:
// without peer access a kernel touching it faults.  Managed memory is
// reachable from every device.
inline int classify_ptr(bool query_ok, int type, int ptr_dev, int cur_dev) {
  if (!query_ok) return PTR_HOST;
  if (type == 2) return ptr_dev == cur_dev ? PTR_DEVICE : PTR_OTHER_DEVICE;
  if (type == 3) return PTR_DEVICE;
  return PTR_HOST;
}

}  // namespace wf
