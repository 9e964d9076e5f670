// probe.cu -- memory-system probes that give the execute kernels' rooflines
// their denominators.
//
// The schemes' work is random record accesses and atomics on control words.
// Two ceilings bound it: bandwidth (HBM sectors, L2 atomics) when the
// records are spread, and latency when hot records serialise their writers,
// since every serializable read-modify-write chain on one record pays the
// round trips of the protocol once per link.  Each probe measures one of
// those quantities on the current GPU with the same PTX memory operations the
// schemes use.
//
// Every loop is bounded: chains by a step count, contended loops by a
// globaltimer deadline, and a lock holder never waits while it holds.
#include <cstring>
#include <string>
#include <vector>

#include "engine.cuh"

namespace gcc {
namespace {

constexpr uint64_t OCC_LOCK_BIT = 1ull << 63;

// ---- dependent chains (one thread) ----------------------------------------
// mode 0: relaxed load, 1: acquire load, 2: atomicAdd(0), 3: failing CAS.
__global__ void chase_kernel(uint64_t* next, uint64_t start, uint32_t steps, int mode,
                             uint64_t* out) {
    uint64_t i = start;
    const uint64_t t0 = globaltimer();
    for (uint32_t s = 0; s < steps; ++s) {
        uint64_t* p = next + i;
        if (mode == 0) i = ld_relaxed(p);
        else if (mode == 1) i = ld_acquire(p);
        else if (mode == 2) i = add64(p, 0ull);
        else i = cas64(p, ~0ull, 0ull);
    }
    const uint64_t t1 = globaltimer();
    out[0] = t1 - t0;
    out[1] = i;
}

// Writes a cyclic chain: word pos[k] holds pos[k + 1].
__global__ void chain_fill_kernel(uint64_t* buf, const uint64_t* pos, uint32_t n) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) buf[pos[k]] = pos[(k + 1) % n];
}

// ---- throughput ------------------------------------------------------------
// CAS on one word per 32-byte sector and thread (always succeeds after the
// first, so every operation modifies its word).
__global__ void cas_distinct_kernel(uint64_t* words, uint32_t iters) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t* p = words + tid * 4;
    uint64_t v = ld_relaxed(p);
    for (uint32_t k = 0; k < iters; ++k) v = cas64(p, v, v + 1) + 1;
    if (v == 0x5a5a5a5a5a5a5a5aull) words[0] = v;
}

// One lane per warp adds to a single word.
__global__ void add_same_kernel(uint64_t* word, uint32_t iters) {
    if ((threadIdx.x & 31) != 0) return;
    for (uint32_t k = 0; k < iters; ++k) add64(word, 1ull);
}

// Random 32-byte sectors (two 16-byte loads of one sector) of a buffer of
// `mask` + 1 sectors, U independent sectors in flight per thread.
template <int U>
__global__ void gather32_kernel(const uint8_t* buf, uint64_t mask, uint32_t iters,
                                uint64_t* sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t acc = 0;
    for (uint32_t k = 0; k < iters; k += U) {
        ulonglong2 v[2 * U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t s = mix64(tid * 0x9E3779B97F4A7C15ull + k + u) & mask;
            v[2 * u] = ld_slot16(buf + s * 32);
            v[2 * u + 1] = ld_slot16(buf + s * 32 + 16);
        }
#pragma unroll
        for (int u = 0; u < 2 * U; ++u) acc += v[u].x ^ v[u].y;
    }
    if (acc == 0x5a5a5a5a5a5a5a5aull) sink[0] = acc;
}

// ---- protocol latencies (one thread, L2-resident lines) --------------------
// mode 0: fence.acq_rel.gpu with nothing outstanding; mode 1: dependent
// acquire-release atomicAdd on one word; mode 2: one uncontended link of the
// OCC commit chain as the execute kernel runs it -- acquire the record's
// version, CAS-lock it, acquire-release commit timestamp, validate one read
// (relaxed load of another word), write the value, release-store the new
// version.  A chain of writers of one record cannot commit faster than one
// such link per writer: each link starts from the previous one's publish.
__global__ void protocol_kernel(uint64_t* ver, uint64_t* val, uint64_t* other,
                                unsigned long long* clock, uint32_t steps, int mode,
                                uint32_t runner, uint64_t* out) {
    // one thread of block `runner` runs; the other blocks only place it on
    // another SM (the latency depends on which die the SM and the words sit on)
    if (blockIdx.x != runner) return;
    uint64_t acc = 0;
    const uint64_t t0 = globaltimer();
    for (uint32_t s = 0; s < steps; ++s) {
        if (mode == 0) {
            fence_acq_rel();
        } else if (mode == 1) {
            unsigned long long b;
            asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                         : "=l"(b) : "l"(clock), "l"(1ull) : "memory");
            acc += b;
        } else {
            const uint64_t v = ld_acquire(ver);
            if (cas64(ver, v, v | OCC_LOCK_BIT) != v) { acc += 1; continue; }
            unsigned long long ts;
            asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                         : "=l"(ts) : "l"(clock), "l"(1ull) : "memory");
            acc += ld_relaxed(other + (ts & 1));
            st_relaxed(val, ts);
            st_release(ver, v + 1);
        }
    }
    const uint64_t t1 = globaltimer();
    out[0] = t1 - t0;
    out[1] = acc;
}

// ---- contended single record (one lane per warp, deadline-bounded) --------
// mode 0: lock hand-off -- test, CAS 0 -> 1, release store 0.
// mode 1: one record under the OCC commit sequence -- acquire the version,
//   read the value, CAS-lock that version, fence, commit ticket, write the
//   value + 1, fence, publish version + 1.  The value must end equal to the
//   number of commits, which checks the sequence itself.
__global__ void contend_kernel(uint64_t* lock, uint64_t* value, unsigned long long* clock,
                               uint64_t budget_ns, int mode, unsigned long long* commits) {
    if ((threadIdx.x & 31) != 0) return;
    const uint64_t end = globaltimer() + budget_ns;
    unsigned long long n = 0;
    while (globaltimer() < end) {
        if (mode == 0) {
            if (ld_relaxed(lock) != 0) continue;
            if (cas64(lock, 0ull, 1ull) != 0ull) continue;
            ++n;
            st_release(lock, 0ull);
        } else {
            const uint64_t v = ld_acquire(lock);
            if (v & OCC_LOCK_BIT) continue;
            const uint64_t x = ld_relaxed(value);
            if (cas64(lock, v, v | OCC_LOCK_BIT) != v) continue;
            fence_acq_rel();
            atomicAdd(clock, 1ull);
            st_relaxed(value, x + 1);
            fence_acq_rel();
            st_relaxed(lock, v + 1);
            ++n;
        }
    }
    atomicAdd(commits, n);
}

struct Ev {
    cudaEvent_t a = nullptr, b = nullptr;
    Ev() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~Ev() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
    float ms() { float m = 0; cudaEventElapsedTime(&m, a, b); return m; }
};

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

uint64_t host_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Distinct random word positions, one per 128-byte line of a buffer of
// `lines` lines, in a random cyclic order (Sattolo's shuffle).
std::vector<uint64_t> random_cycle(uint64_t lines, uint32_t n, uint64_t seed) {
    std::vector<uint64_t> pos(n);
    if (lines == n) {
        for (uint32_t k = 0; k < n; ++k) pos[k] = (uint64_t)k * 16;
    } else {
        const uint64_t stride = lines / n;      // one line per stride window
        for (uint32_t k = 0; k < n; ++k)
            pos[k] = ((uint64_t)k * stride + host_mix(seed + k) % stride) * 16;
    }
    for (uint32_t k = n - 1; k > 0; --k) {
        const uint32_t j = (uint32_t)(host_mix(seed ^ (0xABCDull + k)) % k);
        std::swap(pos[k], pos[j]);
    }
    return pos;
}

}  // namespace
}  // namespace gcc

using namespace gcc;

#define PROBE_CHECK(call)                                                            \
    do {                                                                             \
        const cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                       \
            return set_error(GCC_ERR_CUDA, (std::string(#call) + ": " +              \
                                            cudaGetErrorString(e_)).c_str());        \
    } while (0)

extern "C" gcc_status gcc_probe_memory(int device, gcc_memory_probe* out) {
    if (!out) return set_error(GCC_ERR_INVALID, "gcc_probe_memory: out is NULL");
    std::memset(out, 0, sizeof(*out));
    PROBE_CHECK(cudaSetDevice(device));
    int sms = 0;
    PROBE_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    out->sm_count = (uint32_t)sms;

    constexpr uint64_t BIG = 1ull << 30;           // > L2: HBM-bound gathers and misses
    constexpr uint64_t SMALL = 8ull << 20;         // < L2, > L1: L2-resident chains
    constexpr uint64_t FLUSH = 512ull << 20;       // written to evict L2 before the miss chain
    DevBuf big, small, misc, flush;
    PROBE_CHECK(cudaMalloc(&big.p, BIG));
    PROBE_CHECK(cudaMalloc(&flush.p, FLUSH));
    PROBE_CHECK(cudaMalloc(&small.p, SMALL));
    const uint64_t cas_threads = (uint64_t)sms * 4 * 256;
    const size_t misc_bytes = 4096 + cas_threads * 32;
    PROBE_CHECK(cudaMalloc(&misc.p, misc_bytes));
    PROBE_CHECK(cudaMemset(big.p, 0, BIG));
    PROBE_CHECK(cudaMemset(small.p, 0, SMALL));
    PROBE_CHECK(cudaMemset(misc.p, 0, misc_bytes));
    uint64_t* m64 = static_cast<uint64_t*>(misc.p);
    uint64_t* res = m64;                           // [0, 2): chase results
    uint64_t* lock = m64 + 16;                     // own 128-byte lines
    uint64_t* value = m64 + 32;
    unsigned long long* clock = reinterpret_cast<unsigned long long*>(m64 + 48);
    unsigned long long* commits = reinterpret_cast<unsigned long long*>(m64 + 64);
    uint64_t* one_word = m64 + 80;
    uint64_t* cas_words = m64 + 512;

    // chains: 16384 random lines of the big buffer (misses), all 65536 lines of
    // the small one (L2 hits after a warm pass)
    constexpr uint32_t NBIG = 16384, NSMALL = (uint32_t)(SMALL / 128);
    DevBuf posd;
    PROBE_CHECK(cudaMalloc(&posd.p, (size_t)NSMALL * 8));
    uint64_t big_start = 0;
    {
        const std::vector<uint64_t> pb = random_cycle(BIG / 128, NBIG, 0x51);
        big_start = pb[0];
        PROBE_CHECK(cudaMemcpy(posd.p, pb.data(), pb.size() * 8, cudaMemcpyHostToDevice));
        chain_fill_kernel<<<(NBIG + 255) / 256, 256>>>(static_cast<uint64_t*>(big.p),
                                                       static_cast<uint64_t*>(posd.p), NBIG);
        PROBE_CHECK(cudaGetLastError());
        const std::vector<uint64_t> ps = random_cycle(NSMALL, NSMALL, 0x52);
        PROBE_CHECK(cudaMemcpy(posd.p, ps.data(), ps.size() * 8, cudaMemcpyHostToDevice));
        chain_fill_kernel<<<(NSMALL + 255) / 256, 256>>>(static_cast<uint64_t*>(small.p),
                                                         static_cast<uint64_t*>(posd.p), NSMALL);
        PROBE_CHECK(cudaGetLastError());
    }

    Ev ev;
    // random 32-byte gathers over the big buffer (also evicts the chains'
    // lines from L2 before the miss chain), 4, 8 and 16 sectors in flight per
    // thread at full occupancy; the ceiling is the best of the three
    {
        const uint32_t blocks = (uint32_t)sms * 8, iters = 64;
        const uint8_t* b8 = static_cast<uint8_t*>(big.p);
        const uint64_t mask = BIG / 32 - 1;
        for (int u = 0; u < 3; ++u) {
            auto launch = [&](uint32_t it) {
                if (u == 0) gather32_kernel<4><<<blocks, 256>>>(b8, mask, it, res);
                else if (u == 1) gather32_kernel<8><<<blocks, 256>>>(b8, mask, it, res);
                else gather32_kernel<16><<<blocks, 256>>>(b8, mask, it, res);
            };
            launch(16);
            cudaEventRecord(ev.a);
            launch(iters);
            cudaEventRecord(ev.b);
            PROBE_CHECK(cudaEventSynchronize(ev.b));
            PROBE_CHECK(cudaGetLastError());
            const double gbs = (double)blocks * 256 * iters * 32 / (ev.ms() * 1e-3) / 1e9;
            out->gather32_by_inflight_gbs[u] = gbs;
            if (gbs > out->gather32_gbs) {
                out->gather32_gbs = gbs;
                out->gather32_best_inflight = 4u << u;
            }
        }
    }
    uint64_t h[2];
    auto chase = [&](uint64_t* buf, uint64_t start, uint32_t steps, int mode,
                     double* ns) -> gcc_status {
        chase_kernel<<<1, 1>>>(buf, start, steps, mode, res);
        PROBE_CHECK(cudaMemcpy(h, res, 16, cudaMemcpyDeviceToHost));
        *ns = (double)h[0] / steps;
        return GCC_OK;
    };
    gcc_status s;
    PROBE_CHECK(cudaMemset(flush.p, 1, FLUSH));
    if ((s = chase(static_cast<uint64_t*>(big.p), big_start, 4096, 0, &out->hbm_load_ns)) != GCC_OK) return s;
    double warm = 0;
    uint64_t* sp = static_cast<uint64_t*>(small.p);
    if ((s = chase(sp, 0, NSMALL, 0, &warm)) != GCC_OK) return s;
    if ((s = chase(sp, 0, 32768, 0, &out->l2_load_ns)) != GCC_OK) return s;
    if ((s = chase(sp, 0, 32768, 1, &out->l2_load_acquire_ns)) != GCC_OK) return s;
    if ((s = chase(sp, 0, 32768, 2, &out->l2_atomic_ns)) != GCC_OK) return s;
    if ((s = chase(sp, 0, 32768, 3, &out->l2_cas_ns)) != GCC_OK) return s;

    // protocol latencies on L2-resident words
    {
        uint64_t* ver = m64 + 96;
        uint64_t* val = m64 + 112;
        uint64_t* other = m64 + 128;
        unsigned long long* pclock = reinterpret_cast<unsigned long long*>(m64 + 144);
        double* dst[3] = {&out->fence_ns, &out->atomic_acq_rel_ns, &out->occ_link_ns};
        // eight placements spread over the grid of one block per SM: the
        // least time of each probe, and the greatest of the link
        const uint32_t grid = (uint32_t)sms;
        for (int mode = 0; mode < 3; ++mode) {
            double lo = 0, hi = 0;
            for (uint32_t p = 0; p < 8; ++p) {
                const uint32_t runner = p * grid / 8;
                protocol_kernel<<<grid, 1>>>(ver, val, other, pclock, 256, mode, runner, res);
                protocol_kernel<<<grid, 1>>>(ver, val, other, pclock, 4096, mode, runner, res);
                PROBE_CHECK(cudaMemcpy(h, res, 16, cudaMemcpyDeviceToHost));
                const double ns = (double)h[0] / 4096;
                if (p == 0 || ns < lo) lo = ns;
                if (p == 0 || ns > hi) hi = ns;
            }
            *dst[mode] = lo;
            if (mode == 2) out->occ_link_max_ns = hi;
        }
    }

    // atomic throughput
    {
        const uint32_t blocks = (uint32_t)sms * 4, iters = 64;
        cas_distinct_kernel<<<blocks, 256>>>(cas_words, 4);
        cudaEventRecord(ev.a);
        cas_distinct_kernel<<<blocks, 256>>>(cas_words, iters);
        cudaEventRecord(ev.b);
        PROBE_CHECK(cudaEventSynchronize(ev.b));
        PROBE_CHECK(cudaGetLastError());
        out->cas_distinct_gops = (double)blocks * 256 * iters / (ev.ms() * 1e-3) / 1e9;
    }
    {
        const uint32_t blocks = (uint32_t)sms * 8, iters = 256;
        cudaEventRecord(ev.a);
        add_same_kernel<<<blocks, 256>>>(one_word, iters);
        cudaEventRecord(ev.b);
        PROBE_CHECK(cudaEventSynchronize(ev.b));
        PROBE_CHECK(cudaGetLastError());
        out->add_same_gops = (double)blocks * 8 * iters / (ev.ms() * 1e-3) / 1e9;
    }

    // one contended record, one lane per warp, 20 ms per point: 2 warps on two
    // SMs, 16, one per SM, eight per SM
    out->contenders = (uint32_t)sms * 8;
    constexpr uint64_t BUDGET = 20000000ull;
    const uint32_t grids[4][2] = {{2, 32}, {16, 32}, {(uint32_t)sms, 32}, {(uint32_t)sms, 256}};
    for (int mode = 0; mode < 2; ++mode) {
        double best = 0;
        uint32_t best_n = 0;
        for (const auto& g : grids) {
            PROBE_CHECK(cudaMemset(misc.p, 0, 4096));
            contend_kernel<<<g[0], g[1]>>>(lock, value, clock, BUDGET, mode, commits);
            PROBE_CHECK(cudaDeviceSynchronize());
            unsigned long long n = 0, v = 0;
            PROBE_CHECK(cudaMemcpy(&n, commits, 8, cudaMemcpyDeviceToHost));
            PROBE_CHECK(cudaMemcpy(&v, value, 8, cudaMemcpyDeviceToHost));
            if (n == 0)
                return set_error(GCC_ERR_DEVICE, "gcc_probe_memory: no acquisition in the budget");
            if (mode == 1 && v != n)
                return set_error(GCC_ERR_DEVICE, "gcc_probe_memory: OCC cycle lost an update");
            const double ns = (double)BUDGET / (double)n;
            const uint32_t warps = g[0] * g[1] / 32;
            if (best == 0 || ns < best) { best = ns; best_n = warps; }
            if (mode == 1 && warps == out->contenders) out->occ_cycle_busy_ns = ns;
        }
        if (mode == 0) { out->lock_handoff_ns = best; out->lock_best_contenders = best_n; }
        else { out->occ_cycle_ns = best; out->occ_best_contenders = best_n; }
    }
    return GCC_OK;
}
