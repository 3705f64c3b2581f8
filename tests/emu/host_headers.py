"""Write host-compilable copies of the device headers for the CPU emulation.

core.cuh is copied unchanged except for the helpers written in inline PTX
(acquire load, global timer, release reduction, statistics reduction, cluster
registers and barrier), which are replaced by host equivalents, and the two
time bounds, which are widened for the slower emulation.  Test infrastructure
only: nothing in the library uses this."""
from __future__ import annotations

import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(os.path.dirname(HERE)), "paper_1908_09378_gb300", "csrc")

HOST_VERSIONS = {
    # every caller polls in a spin loop: yield, so that a polling emulated
    # thread leaves its core to the threads it waits for
    "ld_acquire": "__device__ __forceinline__ u64 ld_acquire(const u64 *p)\n{\n"
                  "    std::this_thread::yield();\n"
                  "    return std::atomic_ref<u64>(*const_cast<u64 *>(p)).load(std::memory_order_acquire);\n}\n",
    "gtimer": "__device__ __forceinline__ u64 gtimer()\n{\n    return (u64)std::chrono::duration_cast<"
              "std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch()).count();\n}\n",
    "bar_arrive": "__device__ __forceinline__ void bar_arrive(u64 *p)\n{\n"
                  "    std::atomic_ref<u64>(*p).fetch_add(1, std::memory_order_release);\n}\n",
    "stat_add": "__device__ __forceinline__ void stat_add(u64 *p, u64 v)\n{\n"
                "    std::atomic_ref<u64>(*p).fetch_add(v);\n}\n",
    "cluster_rank": "__device__ __forceinline__ u32 cluster_rank() { return blockIdx.x % g_cluster_size; }\n",
    "cluster_size": "__device__ __forceinline__ u32 cluster_size() { return g_cluster_size; }\n",
    "cluster_barrier": "__device__ __forceinline__ void cluster_barrier() { cluster_sync_at(__LINE__); }\n",
    # bulk copies complete at once on the host
    "smem_u32": "__device__ __forceinline__ u32 smem_u32(const void *) { return 0; }\n",
    "mbar_init": "__device__ __forceinline__ void mbar_init(u64 *) {}\n",
    "mbar_arrive_expect": "__device__ __forceinline__ void mbar_arrive_expect(u64 *, u32) {}\n",
    # a bulk copy needs 16-byte-aligned addresses and a multiple of 16 bytes:
    # the host version checks it, so the emulation catches what would fault
    "bulk_g2s": "__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, u32 bytes, u64 *)\n{\n"
                "    if (((uintptr_t)dst | (uintptr_t)src | bytes) & 15) {\n"
                "        fprintf(stderr, \"bulk copy misaligned: %p %p %u\\n\", dst, src, bytes);\n"
                "        abort();\n    }\n"
                "    std::memcpy(dst, src, bytes);\n}\n",
    "mbar_test": "__device__ __forceinline__ bool mbar_test(u64 *, u32) { return true; }\n",
    # the same offset in the shared memory of CTA `rank` of this cluster
    "dsmem_ld_u64": "__device__ __forceinline__ u64 dsmem_ld_u64(const u64 *local, u32 rank)\n{\n"
                    "    if (g_cluster_size == 1) return *local;\n"
                    "    const unsigned first = blockIdx.x - blockIdx.x % g_cluster_size;\n"
                    "    const size_t off = (const char *)local - (const char *)g_cta_smem[blockIdx.x];\n"
                    "    return std::atomic_ref<u64>(*(u64 *)((char *)g_cta_smem[first + rank] + off))"
                    ".load(std::memory_order_acquire);\n}\n",
    "mbar_inval": "__device__ __forceinline__ void mbar_inval(u64 *) {}\n",
    "fence_proxy_async_global": "__device__ __forceinline__ void fence_proxy_async_global() {}\n",
}


CONCURRENT_HOST_VERSIONS = {
    "st_release": "__device__ __forceinline__ void st_release(u64 *p, u64 v)\n{\n"
                  "    std::atomic_ref<u64>(*p).store(v, std::memory_order_release);\n}\n",
}


def write(out_dir: str) -> None:
    src = open(os.path.join(CSRC, "core.cuh")).read()
    for name, body in HOST_VERSIONS.items():
        m = re.search(r"__device__ __forceinline__ \w+ " + name + r"\(.*?\n\}\n", src, flags=re.S)
        if not m:
            raise RuntimeError(f"device helper {name} not found in core.cuh")
        src = src[:m.start()] + body + src[m.end():]
    src = src.replace("#include <cuda_runtime.h>", '#include "cuda_shim.h"')
    # file-scope shared-memory variables are per CTA: one slot per emulated
    # CTA, selected by the thread's block index
    shared = re.findall(r"^__shared__ ([^;]*?)(\w+);$", src, flags=re.M)
    if not shared:
        raise RuntimeError("no file-scope shared variables found in core.cuh")
    for typ, name in shared:
        src = src.replace(f"__shared__ {typ}{name};",
                          f"inline {typ}g_cta_{name}[512];\n#define {name} g_cta_{name}[blockIdx.x]", 1)
    for old, new in (("constexpr u64 QUERY_NS = 60000000000ull;", "constexpr u64 QUERY_NS = 600000000000ull;"),
                     ("constexpr u64 SPIN_NS = 1000000000ull;", "constexpr u64 SPIN_NS = 60000000000ull;")):
        if old not in src:
            raise RuntimeError(f"time bound not found in core.cuh: {old}")
        src = src.replace(old, new)
    with open(os.path.join(out_dir, "core_host.h"), "w") as f:
        f.write(src)
    conc = open(os.path.join(CSRC, "concurrent.cuh")).read().replace('#include "core.cuh"', '#include "core_host.h"')
    for name, body in CONCURRENT_HOST_VERSIONS.items():
        m = re.search(r"__device__ __forceinline__ \w+ " + name + r"\(.*?\n\}\n", conc, flags=re.S)
        if not m:
            raise RuntimeError(f"device helper {name} not found in concurrent.cuh")
        conc = conc[:m.start()] + body + conc[m.end():]
    with open(os.path.join(out_dir, "concurrent_host.h"), "w") as f:
        f.write(conc)
    heapop = open(os.path.join(CSRC, "heapop.cuh")).read().replace('#include "core.cuh"', '#include "core_host.h"')
    with open(os.path.join(out_dir, "heapop_host.h"), "w") as f:
        f.write(heapop)
    plan = open(os.path.join(CSRC, "plan.h")).read().replace('#include "core.cuh"', '#include "core_host.h"')
    plan = plan.replace('#include "concurrent.cuh"', '#include "concurrent_host.h"')
    with open(os.path.join(out_dir, "plan_host.h"), "w") as f:
        f.write(plan)
    # the records the batched and served kernels read (QueryDesc)
    kern = open(os.path.join(CSRC, "kernels.h")).read()
    for old, new in (("#include <cuda_runtime.h>", '#include "cuda_shim.h"'),
                     ('#include "core.cuh"', '#include "core_host.h"')):
        if old not in kern:
            raise RuntimeError(f"include not found in kernels.h: {old}")
        kern = kern.replace(old, new)
    with open(os.path.join(out_dir, "kernels_host.h"), "w") as f:
        f.write(kern)


def build(name: str, out_dir: str, defines=()) -> str:
    """Write the host headers into out_dir and compile tests/emu/<name>.cpp
    there; returns the executable.  With PBH_EMU_SANITIZE=thread in the
    environment the harness is built with ThreadSanitizer (run it with
    run_env()), which reports any two accesses of one shared-memory word by
    threads of a CTA that no barrier orders, i.e. a read in the same barrier
    interval as another thread's write."""
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if not gxx:
        raise FileNotFoundError("g++ not available")
    write(out_dir)
    exe = os.path.join(out_dir, name)
    flags = ["-O2"]
    if os.environ.get("PBH_EMU_SANITIZE") == "thread":
        flags = ["-O1", "-g", "-fsanitize=thread"]
    res = subprocess.run([gxx, "-std=c++20", *flags, "-pthread", *defines, "-I", out_dir, "-I", HERE, "-o", exe,
                          os.path.join(HERE, name + ".cpp")], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("emulation build failed:\n" + res.stderr[-3000:])
    return exe


def run_env() -> dict:
    """The environment for running a harness: under ThreadSanitizer, the
    suppressions of tests/emu/tsan.supp and a non-zero exit on any other
    report."""
    env = dict(os.environ)
    if env.get("PBH_EMU_SANITIZE") == "thread":
        env["TSAN_OPTIONS"] = (f"suppressions={os.path.join(HERE, 'tsan.supp')} report_signal_unsafe=0 "
                               "history_size=2 exitcode=66")
    return env
