"""Host <-> device bandwidth of this machine's GPU link (GPU report).

The end-to-end figure of the benchmark moves the input from pinned host
memory to the device every step, so that figure is bounded by the link.
This report measures the link three ways, each over 1 GiB (best of five,
CUDA events):
  * copy engines: one pinned buffer copied in 1, 2, 4 and 8 concurrent
    streams;
  * device -> host, one stream;
  * an SM copy kernel (16-byte loads, grid-stride) that reads mapped pinned
    memory through the device pointer cudaHostGetDevicePointer returns.
It prints one JSON line per measurement.

    python tests/report_host_link.py
"""

import ctypes
import json

KERNEL = r'''
#include <cuda_runtime.h>
#include <cstdint>
__global__ void copy16(const uint4* __restrict__ s, uint4* __restrict__ d, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}
void run(long long src, long long dst, long long n16, int blocks, int threads) {
  copy16<<<blocks, threads>>>((const uint4*)src, (uint4*)dst, (size_t)n16);
}
'''


def best_ms(torch, fn, reps=5):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def main():
    import torch
    from torch.utils.cpp_extension import load_inline
    assert torch.cuda.is_available()
    n = 1 << 30
    h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    h.fill_(1)
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    for ns in (1, 2, 4, 8):
        streams = [torch.cuda.Stream() for _ in range(ns)]

        def up():
            cur = torch.cuda.current_stream()
            part = n // ns
            for i, s in enumerate(streams):
                s.wait_stream(cur)
                with torch.cuda.stream(s):
                    d[i * part:(i + 1) * part].copy_(h[i * part:(i + 1) * part], non_blocking=True)
            for s in streams:
                cur.wait_stream(s)
        ms = best_ms(torch, up)
        print(json.dumps({"path": "h2d copy engines", "streams": ns, "GB/s": n / ms / 1e6}), flush=True)
    ms = best_ms(torch, lambda: h.copy_(d, non_blocking=True))
    print(json.dumps({"path": "d2h copy engine", "streams": 1, "GB/s": n / ms / 1e6}), flush=True)

    mod = load_inline("report_host_link_copy", cpp_sources="void run(long long, long long, long long, int, int);",
                      cuda_sources=KERNEL, functions=["run"],
                      extra_cuda_cflags=["-gencode", "arch=compute_103a,code=sm_103a", "-O3"])
    rt = ctypes.CDLL("libcudart.so.13")
    hm = ctypes.c_void_p()
    if rt.cudaHostAlloc(ctypes.byref(hm), ctypes.c_size_t(n), ctypes.c_uint(2)) != 0:   # mapped
        raise RuntimeError("cudaHostAlloc(mapped) failed")
    try:
        dp = ctypes.c_void_p()
        if rt.cudaHostGetDevicePointer(ctypes.byref(dp), hm, ctypes.c_uint(0)) != 0:
            raise RuntimeError("cudaHostGetDevicePointer failed")
        ctypes.memset(hm, 1, n)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        for blocks, threads in ((sms, 1024), (2 * sms, 1024), (8 * sms, 256)):
            ms = best_ms(torch, lambda: mod.run(dp.value, d.data_ptr(), n // 16, blocks, threads))
            print(json.dumps({"path": "h2d SM copy kernel (mapped pinned memory)",
                              "grid": blocks, "block": threads, "GB/s": n / ms / 1e6}), flush=True)
    finally:
        rt.cudaFreeHost(hm)


if __name__ == "__main__":
    main()
