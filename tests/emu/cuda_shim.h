// Host emulation of the CUDA constructs the device code uses, for running the
// kernels' control flow on the CPU in tests: every CUDA thread is a
// std::thread, __syncthreads is a per-CTA std::barrier, warp shuffles and
// ballots are a per-warp exchange with a warp barrier, global atomics are
// std::atomic_ref.  Shared memory is a separate allocation per emulated CTA.
// Test infrastructure only.
#pragma once
#include <algorithm>
#include <atomic>
#include <barrier>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>

struct uint3_ { unsigned x = 0, y = 0, z = 0; };
inline thread_local uint3_ threadIdx;
inline thread_local uint3_ blockIdx;
inline uint3_ gridDim{1, 1, 1};
inline uint3_ blockDim{256, 1, 1};

#define __device__
#define __global__
#define __host__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
#define __launch_bounds__(...)
#define __shared__
#define __align__(n) alignas(n)

inline thread_local std::barrier<> *g_cta_bar = nullptr;
inline thread_local int g_gid = 0; // emulated thread's index over all CTAs (diagnostics)
inline int g_site_line[1 << 17]; // per emulated thread (up to 512 CTAs)
inline unsigned long long g_site_count[1 << 17];
inline std::atomic<unsigned long long> g_progress{0};
inline int g_hist[1 << 17][8];
inline int g_hpos[1 << 17];
inline void sync_at(int line)
{
    g_hist[g_gid][g_hpos[g_gid]++ & 7] = line;
    g_site_line[g_gid] = line;
    g_site_count[g_gid]++;
    g_progress.fetch_add(1, std::memory_order_relaxed);
    g_cta_bar->arrive_and_wait();
    g_site_line[g_gid] = -line;
}
#define __syncthreads() sync_at(__LINE__)

// Thread-block clusters: the emulated launch sets the cluster size, each
// thread its cluster's barrier (all threads of all CTAs of the cluster, as
// the hardware cluster barrier is) and the table of every CTA's shared
// memory, through which distributed shared memory is read.  With a cluster
// size of 1 the cluster barrier is the CTA's.
inline unsigned g_cluster_size = 1;
inline thread_local std::barrier<> *g_cluster_bar = nullptr;
inline void *g_cta_smem[512];
inline void cluster_sync_at(int line)
{
    if (!g_cluster_bar) {
        sync_at(line);
        return;
    }
    g_hist[g_gid][g_hpos[g_gid]++ & 7] = 200000 + line;
    g_site_line[g_gid] = 200000 + line;
    g_site_count[g_gid]++;
    g_progress.fetch_add(1, std::memory_order_relaxed);
    g_cluster_bar->arrive_and_wait();
    g_site_line[g_gid] = -(200000 + line);
}
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void __threadfence_block() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void __threadfence_system() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void __nanosleep(unsigned) { std::this_thread::yield(); }

struct WarpX {
    std::barrier<> *bar;
    unsigned long long v[32];
};
inline WarpX g_warps[32];
inline thread_local WarpX *g_wx = g_warps; // this CTA's warp exchange table

inline unsigned long long warp_exchange(unsigned long long mine, int src)
{
    g_progress.fetch_add(1, std::memory_order_relaxed);
    g_site_line[g_gid] = 100000;
    WarpX &w = g_wx[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    w.v[lane] = mine;
    w.bar->arrive_and_wait();
    unsigned long long r = w.v[src & 31];
    w.bar->arrive_and_wait();
    return r;
}
template <class T> T __shfl_sync(unsigned, T v, int src) { return (T)warp_exchange((unsigned long long)v, src); }
template <class T> T __shfl_up_sync(unsigned, T v, unsigned d)
{
    const int lane = threadIdx.x & 31;
    const int src = lane - (int)d;
    T r = (T)warp_exchange((unsigned long long)v, src < 0 ? lane : src);
    return r;
}
template <class T> T __shfl_xor_sync(unsigned, T v, int m)
{
    return (T)warp_exchange((unsigned long long)v, (threadIdx.x & 31) ^ m);
}
inline unsigned __ballot_sync(unsigned, bool p)
{
    g_progress.fetch_add(1, std::memory_order_relaxed);
    g_site_line[g_gid] = 200000;
    WarpX &w = g_wx[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    w.v[lane] = p ? 1 : 0;
    w.bar->arrive_and_wait();
    unsigned m = 0;
    for (int i = 0; i < 32; i++) m |= (w.v[i] ? 1u : 0u) << i;
    w.bar->arrive_and_wait();
    return m;
}
inline int __popc(unsigned x) { return __builtin_popcount(x); }

inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v)
{
    return std::atomic_ref<unsigned long long>(*p).fetch_add(v);
}
inline unsigned atomicAdd(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_add(v); }
inline unsigned long long atomicMin(unsigned long long *p, unsigned long long v)
{
    std::atomic_ref<unsigned long long> a(*p);
    unsigned long long old = a.load();
    while (old > v && !a.compare_exchange_weak(old, v)) {
    }
    return old;
}
inline unsigned long long atomicMax(unsigned long long *p, unsigned long long v)
{
    std::atomic_ref<unsigned long long> a(*p);
    unsigned long long old = a.load();
    while (old < v && !a.compare_exchange_weak(old, v)) {
    }
    return old;
}
inline unsigned atomicExch(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).exchange(v); }
inline unsigned long long atomicExch(unsigned long long *p, unsigned long long v)
{
    return std::atomic_ref<unsigned long long>(*p).exchange(v);
}
inline unsigned atomicCAS(unsigned *p, unsigned cmp, unsigned val)
{
    std::atomic_ref<unsigned> a(*p);
    a.compare_exchange_strong(cmp, val);
    return cmp;
}
template <class T> T __ldg(const T *p) { return *p; }
inline unsigned long long __ldcg(const unsigned long long *p)
{
    return std::atomic_ref<unsigned long long>(*const_cast<unsigned long long *>(p)).load(std::memory_order_relaxed);
}
inline unsigned __ldcg(const unsigned *p)
{
    return std::atomic_ref<unsigned>(*const_cast<unsigned *>(p)).load(std::memory_order_relaxed);
}
template <class T> inline T min(T a, T b) { return a < b ? a : b; }
template <class T> inline T max(T a, T b) { return a < b ? b : a; }
inline unsigned long long atomicOr(unsigned long long *p, unsigned long long v)
{
    return std::atomic_ref<unsigned long long>(*p).fetch_or(v);
}
inline unsigned atomicOr(unsigned *p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_or(v); }
inline unsigned atomicMax(unsigned *p, unsigned v)
{
    std::atomic_ref<unsigned> a(*p);
    unsigned old = a.load();
    while (old < v && !a.compare_exchange_weak(old, v)) {
    }
    return old;
}
