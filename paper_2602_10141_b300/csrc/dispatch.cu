// Runtime-n dispatch to the compile-time-n kernels (written by build.py).
#include "common.cuh"

namespace permx {

cudaError_t dispatch_modp(int n, const ModpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    // blocks of kRyserThreads threads while the launch fills every SM; a
    // smaller launch takes smaller blocks (down to one warp) so that its
    // warps spread over more SMs instead of sharing a few (the results do
    // not depend on the block size)
    int threads = kRyserThreads;
    auto grid_for = [&](int bps, int lanes_per_item = 1) {
        const uint64_t lanes = items * lanes_per_item;
        const uint64_t sms = (uint64_t)sm_count();
        while (threads > 32 && (lanes + threads - 1) / threads < sms) threads >>= 1;
        uint64_t want = (lanes + threads - 1) / threads;
        uint64_t cap = sms * (uint64_t)bps * (uint64_t)(kRyserThreads / threads);
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: { const int g = grid_for(blocks_per_sm_modp<1>(), 1); return launch_modp<1>(L, g, threads, s); }
        case 2: { const int g = grid_for(blocks_per_sm_modp<2>(), 1); return launch_modp<2>(L, g, threads, s); }
        case 3: { const int g = grid_for(blocks_per_sm_modp<3>(), 1); return launch_modp<3>(L, g, threads, s); }
        case 4: { const int g = grid_for(blocks_per_sm_modp<4>(), 1); return launch_modp<4>(L, g, threads, s); }
        case 5: { const int g = grid_for(blocks_per_sm_modp<5>(), 1); return launch_modp<5>(L, g, threads, s); }
        case 6: { const int g = grid_for(blocks_per_sm_modp<6>(), 1); return launch_modp<6>(L, g, threads, s); }
        case 7: { const int g = grid_for(blocks_per_sm_modp<7>(), 1); return launch_modp<7>(L, g, threads, s); }
        case 8: { const int g = grid_for(blocks_per_sm_modp<8>(), 1); return launch_modp<8>(L, g, threads, s); }
        case 9: { const int g = grid_for(blocks_per_sm_modp<9>(), 1); return launch_modp<9>(L, g, threads, s); }
        case 10: { const int g = grid_for(blocks_per_sm_modp<10>(), 1); return launch_modp<10>(L, g, threads, s); }
        case 11: { const int g = grid_for(blocks_per_sm_modp<11>(), 1); return launch_modp<11>(L, g, threads, s); }
        case 12: { const int g = grid_for(blocks_per_sm_modp<12>(), 1); return launch_modp<12>(L, g, threads, s); }
        case 13: { const int g = grid_for(blocks_per_sm_modp<13>(), 1); return launch_modp<13>(L, g, threads, s); }
        case 14: { const int g = grid_for(blocks_per_sm_modp<14>(), 1); return launch_modp<14>(L, g, threads, s); }
        case 15: { const int g = grid_for(blocks_per_sm_modp<15>(), 1); return launch_modp<15>(L, g, threads, s); }
        case 16: { const int g = grid_for(blocks_per_sm_modp<16>(), 1); return launch_modp<16>(L, g, threads, s); }
        case 17: { const int g = grid_for(blocks_per_sm_modp<17>(), 1); return launch_modp<17>(L, g, threads, s); }
        case 18: { const int g = grid_for(blocks_per_sm_modp<18>(), 1); return launch_modp<18>(L, g, threads, s); }
        case 19: { const int g = grid_for(blocks_per_sm_modp<19>(), 1); return launch_modp<19>(L, g, threads, s); }
        case 20: { const int g = grid_for(blocks_per_sm_modp<20>(), 1); return launch_modp<20>(L, g, threads, s); }
        case 21: { const int g = grid_for(blocks_per_sm_modp<21>(), 1); return launch_modp<21>(L, g, threads, s); }
        case 22: { const int g = grid_for(blocks_per_sm_modp<22>(), 1); return launch_modp<22>(L, g, threads, s); }
        case 23: { const int g = grid_for(blocks_per_sm_modp<23>(), 1); return launch_modp<23>(L, g, threads, s); }
        case 24: { const int g = grid_for(blocks_per_sm_modp<24>(), 1); return launch_modp<24>(L, g, threads, s); }
        case 25: { const int g = grid_for(blocks_per_sm_modp<25>(), 1); return launch_modp<25>(L, g, threads, s); }
        case 26: { const int g = grid_for(blocks_per_sm_modp<26>(), 1); return launch_modp<26>(L, g, threads, s); }
        case 27: { const int g = grid_for(blocks_per_sm_modp<27>(), 1); return launch_modp<27>(L, g, threads, s); }
        case 28: { const int g = grid_for(blocks_per_sm_modp<28>(), 1); return launch_modp<28>(L, g, threads, s); }
        case 29: { const int g = grid_for(blocks_per_sm_modp<29>(), 1); return launch_modp<29>(L, g, threads, s); }
        case 30: { const int g = grid_for(blocks_per_sm_modp<30>(), 1); return launch_modp<30>(L, g, threads, s); }
        case 31: { const int g = grid_for(blocks_per_sm_modp<31>(), 1); return launch_modp<31>(L, g, threads, s); }
        case 32: { const int g = grid_for(blocks_per_sm_modp<32>(), 1); return launch_modp<32>(L, g, threads, s); }
        case 33: { const int g = grid_for(blocks_per_sm_modp<33>(), 1); return launch_modp<33>(L, g, threads, s); }
        case 34: { const int g = grid_for(blocks_per_sm_modp<34>(), 1); return launch_modp<34>(L, g, threads, s); }
        case 35: { const int g = grid_for(blocks_per_sm_modp<35>(), 1); return launch_modp<35>(L, g, threads, s); }
        case 36: { const int g = grid_for(blocks_per_sm_modp<36>(), 1); return launch_modp<36>(L, g, threads, s); }
        case 37: { const int g = grid_for(blocks_per_sm_modp<37>(), 1); return launch_modp<37>(L, g, threads, s); }
        case 38: { const int g = grid_for(blocks_per_sm_modp<38>(), 1); return launch_modp<38>(L, g, threads, s); }
        case 39: { const int g = grid_for(blocks_per_sm_modp<39>(), 1); return launch_modp<39>(L, g, threads, s); }
        case 40: { const int g = grid_for(blocks_per_sm_modp<40>(), 1); return launch_modp<40>(L, g, threads, s); }
        case 41: { const int g = grid_for(blocks_per_sm_modp<41>(), 1); return launch_modp<41>(L, g, threads, s); }
        case 42: { const int g = grid_for(blocks_per_sm_modp<42>(), 1); return launch_modp<42>(L, g, threads, s); }
        case 43: { const int g = grid_for(blocks_per_sm_modp<43>(), 1); return launch_modp<43>(L, g, threads, s); }
        case 44: { const int g = grid_for(blocks_per_sm_modp<44>(), 1); return launch_modp<44>(L, g, threads, s); }
        case 45: { const int g = grid_for(blocks_per_sm_modp<45>(), 1); return launch_modp<45>(L, g, threads, s); }
        case 46: { const int g = grid_for(blocks_per_sm_modp<46>(), 1); return launch_modp<46>(L, g, threads, s); }
        case 47: { const int g = grid_for(blocks_per_sm_modp<47>(), 1); return launch_modp<47>(L, g, threads, s); }
        case 48: { const int g = grid_for(blocks_per_sm_modp<48>(), 1); return launch_modp<48>(L, g, threads, s); }
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_f64(int n, const FpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    // blocks of kRyserThreads threads while the launch fills every SM; a
    // smaller launch takes smaller blocks (down to one warp) so that its
    // warps spread over more SMs instead of sharing a few (the results do
    // not depend on the block size)
    int threads = kRyserThreads;
    auto grid_for = [&](int bps, int lanes_per_item = 1) {
        const uint64_t lanes = items * lanes_per_item;
        const uint64_t sms = (uint64_t)sm_count();
        while (threads > 32 && (lanes + threads - 1) / threads < sms) threads >>= 1;
        uint64_t want = (lanes + threads - 1) / threads;
        uint64_t cap = sms * (uint64_t)bps * (uint64_t)(kRyserThreads / threads);
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: { const int g = grid_for(blocks_per_sm_f64<1>(), 1); return launch_f64<1>(L, g, threads, s); }
        case 2: { const int g = grid_for(blocks_per_sm_f64<2>(), 1); return launch_f64<2>(L, g, threads, s); }
        case 3: { const int g = grid_for(blocks_per_sm_f64<3>(), 1); return launch_f64<3>(L, g, threads, s); }
        case 4: { const int g = grid_for(blocks_per_sm_f64<4>(), 1); return launch_f64<4>(L, g, threads, s); }
        case 5: { const int g = grid_for(blocks_per_sm_f64<5>(), 1); return launch_f64<5>(L, g, threads, s); }
        case 6: { const int g = grid_for(blocks_per_sm_f64<6>(), 1); return launch_f64<6>(L, g, threads, s); }
        case 7: { const int g = grid_for(blocks_per_sm_f64<7>(), 1); return launch_f64<7>(L, g, threads, s); }
        case 8: { const int g = grid_for(blocks_per_sm_f64<8>(), 1); return launch_f64<8>(L, g, threads, s); }
        case 9: { const int g = grid_for(blocks_per_sm_f64<9>(), 1); return launch_f64<9>(L, g, threads, s); }
        case 10: { const int g = grid_for(blocks_per_sm_f64<10>(), 1); return launch_f64<10>(L, g, threads, s); }
        case 11: { const int g = grid_for(blocks_per_sm_f64<11>(), 1); return launch_f64<11>(L, g, threads, s); }
        case 12: { const int g = grid_for(blocks_per_sm_f64<12>(), 1); return launch_f64<12>(L, g, threads, s); }
        case 13: { const int g = grid_for(blocks_per_sm_f64<13>(), 1); return launch_f64<13>(L, g, threads, s); }
        case 14: { const int g = grid_for(blocks_per_sm_f64<14>(), 1); return launch_f64<14>(L, g, threads, s); }
        case 15: { const int g = grid_for(blocks_per_sm_f64<15>(), 1); return launch_f64<15>(L, g, threads, s); }
        case 16: { const int g = grid_for(blocks_per_sm_f64<16>(), 1); return launch_f64<16>(L, g, threads, s); }
        case 17: { const int g = grid_for(blocks_per_sm_f64<17>(), 1); return launch_f64<17>(L, g, threads, s); }
        case 18: { const int g = grid_for(blocks_per_sm_f64<18>(), 1); return launch_f64<18>(L, g, threads, s); }
        case 19: { const int g = grid_for(blocks_per_sm_f64<19>(), 1); return launch_f64<19>(L, g, threads, s); }
        case 20: { const int g = grid_for(blocks_per_sm_f64<20>(), 1); return launch_f64<20>(L, g, threads, s); }
        case 21: { const int g = grid_for(blocks_per_sm_f64<21>(), 1); return launch_f64<21>(L, g, threads, s); }
        case 22: { const int g = grid_for(blocks_per_sm_f64<22>(), 1); return launch_f64<22>(L, g, threads, s); }
        case 23: { const int g = grid_for(blocks_per_sm_f64<23>(), 1); return launch_f64<23>(L, g, threads, s); }
        case 24: { const int g = grid_for(blocks_per_sm_f64<24>(), 1); return launch_f64<24>(L, g, threads, s); }
        case 25: { const int g = grid_for(blocks_per_sm_f64<25>(), 1); return launch_f64<25>(L, g, threads, s); }
        case 26: { const int g = grid_for(blocks_per_sm_f64<26>(), 1); return launch_f64<26>(L, g, threads, s); }
        case 27: { const int g = grid_for(blocks_per_sm_f64<27>(), 1); return launch_f64<27>(L, g, threads, s); }
        case 28: { const int g = grid_for(blocks_per_sm_f64<28>(), 1); return launch_f64<28>(L, g, threads, s); }
        case 29: { const int g = grid_for(blocks_per_sm_f64<29>(), 1); return launch_f64<29>(L, g, threads, s); }
        case 30: { const int g = grid_for(blocks_per_sm_f64<30>(), 1); return launch_f64<30>(L, g, threads, s); }
        case 31: { const int g = grid_for(blocks_per_sm_f64<31>(), 1); return launch_f64<31>(L, g, threads, s); }
        case 32: { const int g = grid_for(blocks_per_sm_f64<32>(), 1); return launch_f64<32>(L, g, threads, s); }
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_c128(int n, const FpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    // blocks of kRyserThreads threads while the launch fills every SM; a
    // smaller launch takes smaller blocks (down to one warp) so that its
    // warps spread over more SMs instead of sharing a few (the results do
    // not depend on the block size)
    int threads = kRyserThreads;
    auto grid_for = [&](int bps, int lanes_per_item = 1) {
        const uint64_t lanes = items * lanes_per_item;
        const uint64_t sms = (uint64_t)sm_count();
        while (threads > 32 && (lanes + threads - 1) / threads < sms) threads >>= 1;
        uint64_t want = (lanes + threads - 1) / threads;
        uint64_t cap = sms * (uint64_t)bps * (uint64_t)(kRyserThreads / threads);
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: { const int g = grid_for(blocks_per_sm_c128<1>(), 1); return launch_c128<1>(L, g, threads, s); }
        case 2: { const int g = grid_for(blocks_per_sm_c128<2>(), 1); return launch_c128<2>(L, g, threads, s); }
        case 3: { const int g = grid_for(blocks_per_sm_c128<3>(), 1); return launch_c128<3>(L, g, threads, s); }
        case 4: { const int g = grid_for(blocks_per_sm_c128<4>(), 1); return launch_c128<4>(L, g, threads, s); }
        case 5: { const int g = grid_for(blocks_per_sm_c128<5>(), 1); return launch_c128<5>(L, g, threads, s); }
        case 6: { const int g = grid_for(blocks_per_sm_c128<6>(), 1); return launch_c128<6>(L, g, threads, s); }
        case 7: { const int g = grid_for(blocks_per_sm_c128<7>(), 1); return launch_c128<7>(L, g, threads, s); }
        case 8: { const int g = grid_for(blocks_per_sm_c128<8>(), 1); return launch_c128<8>(L, g, threads, s); }
        case 9: { const int g = grid_for(blocks_per_sm_c128<9>(), 1); return launch_c128<9>(L, g, threads, s); }
        case 10: { const int g = grid_for(blocks_per_sm_c128<10>(), 1); return launch_c128<10>(L, g, threads, s); }
        case 11: { const int g = grid_for(blocks_per_sm_c128<11>(), 1); return launch_c128<11>(L, g, threads, s); }
        case 12: { const int g = grid_for(blocks_per_sm_c128<12>(), 1); return launch_c128<12>(L, g, threads, s); }
        case 13: { const int g = grid_for(blocks_per_sm_c128<13>(), 1); return launch_c128<13>(L, g, threads, s); }
        case 14: { const int g = grid_for(blocks_per_sm_c128<14>(), 1); return launch_c128<14>(L, g, threads, s); }
        case 15: { const int g = grid_for(blocks_per_sm_c128<15>(), 1); return launch_c128<15>(L, g, threads, s); }
        case 16: { const int g = grid_for(blocks_per_sm_c128<16>(), 1); return launch_c128<16>(L, g, threads, s); }
        case 17: { const int g = grid_for(blocks_per_sm_c128<17>(), 1); return launch_c128<17>(L, g, threads, s); }
        case 18: { const int g = grid_for(blocks_per_sm_c128<18>(), 1); return launch_c128<18>(L, g, threads, s); }
        case 19: { const int g = grid_for(blocks_per_sm_c128<19>(), 1); return launch_c128<19>(L, g, threads, s); }
        case 20: { const int g = grid_for(blocks_per_sm_c128<20>(), 1); return launch_c128<20>(L, g, threads, s); }
        case 21: { const int g = grid_for(blocks_per_sm_c128<21>(), 1); return launch_c128<21>(L, g, threads, s); }
        case 22: { const int g = grid_for(blocks_per_sm_c128<22>(), 1); return launch_c128<22>(L, g, threads, s); }
        case 23: { const int g = grid_for(blocks_per_sm_c128<23>(), 1); return launch_c128<23>(L, g, threads, s); }
        case 24: { const int g = grid_for(blocks_per_sm_c128<24>(), 1); return launch_c128<24>(L, g, threads, s); }
        case 25: { const int g = grid_for(blocks_per_sm_c128<25>(), 1); return launch_c128<25>(L, g, threads, s); }
        case 26: { const int g = grid_for(blocks_per_sm_c128<26>(), 1); return launch_c128<26>(L, g, threads, s); }
        case 27: { const int g = grid_for(blocks_per_sm_c128<27>(), 1); return launch_c128<27>(L, g, threads, s); }
        case 28: { const int g = grid_for(blocks_per_sm_c128<28>(), 1); return launch_c128<28>(L, g, threads, s); }
        case 29: { const int g = grid_for(blocks_per_sm_c128<29>(), 1); return launch_c128<29>(L, g, threads, s); }
        case 30: { const int g = grid_for(blocks_per_sm_c128<30>(), 1); return launch_c128<30>(L, g, threads, s); }
        case 31: { const int g = grid_for(blocks_per_sm_c128<31>(), 1); return launch_c128<31>(L, g, threads, s); }
        case 32: { const int g = grid_for(blocks_per_sm_c128<32>(), 1); return launch_c128<32>(L, g, threads, s); }
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_x64r(int n, const FpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    // blocks of kRyserThreads threads while the launch fills every SM; a
    // smaller launch takes smaller blocks (down to one warp) so that its
    // warps spread over more SMs instead of sharing a few (the results do
    // not depend on the block size)
    int threads = kRyserThreads;
    auto grid_for = [&](int bps, int lanes_per_item = 1) {
        const uint64_t lanes = items * lanes_per_item;
        const uint64_t sms = (uint64_t)sm_count();
        while (threads > 32 && (lanes + threads - 1) / threads < sms) threads >>= 1;
        uint64_t want = (lanes + threads - 1) / threads;
        uint64_t cap = sms * (uint64_t)bps * (uint64_t)(kRyserThreads / threads);
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: { const int g = grid_for(blocks_per_sm_x64r<1>(), 1); return launch_x64r<1>(L, g, threads, s); }
        case 2: { const int g = grid_for(blocks_per_sm_x64r<2>(), 1); return launch_x64r<2>(L, g, threads, s); }
        case 3: { const int g = grid_for(blocks_per_sm_x64r<3>(), 1); return launch_x64r<3>(L, g, threads, s); }
        case 4: { const int g = grid_for(blocks_per_sm_x64r<4>(), 1); return launch_x64r<4>(L, g, threads, s); }
        case 5: { const int g = grid_for(blocks_per_sm_x64r<5>(), 1); return launch_x64r<5>(L, g, threads, s); }
        case 6: { const int g = grid_for(blocks_per_sm_x64r<6>(), 1); return launch_x64r<6>(L, g, threads, s); }
        case 7: { const int g = grid_for(blocks_per_sm_x64r<7>(), 1); return launch_x64r<7>(L, g, threads, s); }
        case 8: { const int g = grid_for(blocks_per_sm_x64r<8>(), 1); return launch_x64r<8>(L, g, threads, s); }
        case 9: { const int g = grid_for(blocks_per_sm_x64r<9>(), 1); return launch_x64r<9>(L, g, threads, s); }
        case 10: { const int g = grid_for(blocks_per_sm_x64r<10>(), 1); return launch_x64r<10>(L, g, threads, s); }
        case 11: { const int g = grid_for(blocks_per_sm_x64r<11>(), 1); return launch_x64r<11>(L, g, threads, s); }
        case 12: { const int g = grid_for(blocks_per_sm_x64r<12>(), 1); return launch_x64r<12>(L, g, threads, s); }
        case 13: { const int g = grid_for(blocks_per_sm_x64r<13>(), 1); return launch_x64r<13>(L, g, threads, s); }
        case 14: { const int g = grid_for(blocks_per_sm_x64r<14>(), 1); return launch_x64r<14>(L, g, threads, s); }
        case 15: { const int g = grid_for(blocks_per_sm_x64r<15>(), 1); return launch_x64r<15>(L, g, threads, s); }
        case 16: { const int g = grid_for(blocks_per_sm_x64r<16>(), 1); return launch_x64r<16>(L, g, threads, s); }
        case 17: { const int g = grid_for(blocks_per_sm_x64r<17>(), 1); return launch_x64r<17>(L, g, threads, s); }
        case 18: { const int g = grid_for(blocks_per_sm_x64r<18>(), 1); return launch_x64r<18>(L, g, threads, s); }
        case 19: { const int g = grid_for(blocks_per_sm_x64r<19>(), 1); return launch_x64r<19>(L, g, threads, s); }
        case 20: { const int g = grid_for(blocks_per_sm_x64r<20>(), 1); return launch_x64r<20>(L, g, threads, s); }
        case 21: { const int g = grid_for(blocks_per_sm_x64r<21>(), 1); return launch_x64r<21>(L, g, threads, s); }
        case 22: { const int g = grid_for(blocks_per_sm_x64r<22>(), 1); return launch_x64r<22>(L, g, threads, s); }
        case 23: { const int g = grid_for(blocks_per_sm_x64r<23>(), 1); return launch_x64r<23>(L, g, threads, s); }
        case 24: { const int g = grid_for(blocks_per_sm_x64r<24>(), 1); return launch_x64r<24>(L, g, threads, s); }
        case 25: { const int g = grid_for(blocks_per_sm_x64r<25>(), 1); return launch_x64r<25>(L, g, threads, s); }
        case 26: { const int g = grid_for(blocks_per_sm_x64r<26>(), 1); return launch_x64r<26>(L, g, threads, s); }
        case 27: { const int g = grid_for(blocks_per_sm_x64r<27>(), 1); return launch_x64r<27>(L, g, threads, s); }
        case 28: { const int g = grid_for(blocks_per_sm_x64r<28>(), 1); return launch_x64r<28>(L, g, threads, s); }
        case 29: { const int g = grid_for(blocks_per_sm_x64r<29>(), 1); return launch_x64r<29>(L, g, threads, s); }
        case 30: { const int g = grid_for(blocks_per_sm_x64r<30>(), 1); return launch_x64r<30>(L, g, threads, s); }
        case 31: { const int g = grid_for(blocks_per_sm_x64r<31>(), 1); return launch_x64r<31>(L, g, threads, s); }
        case 32: { const int g = grid_for(blocks_per_sm_x64r<32>(), 1); return launch_x64r<32>(L, g, threads, s); }
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_x64c(int n, const FpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    // blocks of kRyserThreads threads while the launch fills every SM; a
    // smaller launch takes smaller blocks (down to one warp) so that its
    // warps spread over more SMs instead of sharing a few (the results do
    // not depend on the block size)
    int threads = kRyserThreads;
    auto grid_for = [&](int bps, int lanes_per_item = 1) {
        const uint64_t lanes = items * lanes_per_item;
        const uint64_t sms = (uint64_t)sm_count();
        while (threads > 32 && (lanes + threads - 1) / threads < sms) threads >>= 1;
        uint64_t want = (lanes + threads - 1) / threads;
        uint64_t cap = sms * (uint64_t)bps * (uint64_t)(kRyserThreads / threads);
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: { const int g = grid_for(blocks_per_sm_x64c<1>(), x64c_paired(1) ? 2 : 1); return launch_x64c<1>(L, g, threads, s); }
        case 2: { const int g = grid_for(blocks_per_sm_x64c<2>(), x64c_paired(2) ? 2 : 1); return launch_x64c<2>(L, g, threads, s); }
        case 3: { const int g = grid_for(blocks_per_sm_x64c<3>(), x64c_paired(3) ? 2 : 1); return launch_x64c<3>(L, g, threads, s); }
        case 4: { const int g = grid_for(blocks_per_sm_x64c<4>(), x64c_paired(4) ? 2 : 1); return launch_x64c<4>(L, g, threads, s); }
        case 5: { const int g = grid_for(blocks_per_sm_x64c<5>(), x64c_paired(5) ? 2 : 1); return launch_x64c<5>(L, g, threads, s); }
        case 6: { const int g = grid_for(blocks_per_sm_x64c<6>(), x64c_paired(6) ? 2 : 1); return launch_x64c<6>(L, g, threads, s); }
        case 7: { const int g = grid_for(blocks_per_sm_x64c<7>(), x64c_paired(7) ? 2 : 1); return launch_x64c<7>(L, g, threads, s); }
        case 8: { const int g = grid_for(blocks_per_sm_x64c<8>(), x64c_paired(8) ? 2 : 1); return launch_x64c<8>(L, g, threads, s); }
        case 9: { const int g = grid_for(blocks_per_sm_x64c<9>(), x64c_paired(9) ? 2 : 1); return launch_x64c<9>(L, g, threads, s); }
        case 10: { const int g = grid_for(blocks_per_sm_x64c<10>(), x64c_paired(10) ? 2 : 1); return launch_x64c<10>(L, g, threads, s); }
        case 11: { const int g = grid_for(blocks_per_sm_x64c<11>(), x64c_paired(11) ? 2 : 1); return launch_x64c<11>(L, g, threads, s); }
        case 12: { const int g = grid_for(blocks_per_sm_x64c<12>(), x64c_paired(12) ? 2 : 1); return launch_x64c<12>(L, g, threads, s); }
        case 13: { const int g = grid_for(blocks_per_sm_x64c<13>(), x64c_paired(13) ? 2 : 1); return launch_x64c<13>(L, g, threads, s); }
        case 14: { const int g = grid_for(blocks_per_sm_x64c<14>(), x64c_paired(14) ? 2 : 1); return launch_x64c<14>(L, g, threads, s); }
        case 15: { const int g = grid_for(blocks_per_sm_x64c<15>(), x64c_paired(15) ? 2 : 1); return launch_x64c<15>(L, g, threads, s); }
        case 16: { const int g = grid_for(blocks_per_sm_x64c<16>(), x64c_paired(16) ? 2 : 1); return launch_x64c<16>(L, g, threads, s); }
        case 17: { const int g = grid_for(blocks_per_sm_x64c<17>(), x64c_paired(17) ? 2 : 1); return launch_x64c<17>(L, g, threads, s); }
        case 18: { const int g = grid_for(blocks_per_sm_x64c<18>(), x64c_paired(18) ? 2 : 1); return launch_x64c<18>(L, g, threads, s); }
        case 19: { const int g = grid_for(blocks_per_sm_x64c<19>(), x64c_paired(19) ? 2 : 1); return launch_x64c<19>(L, g, threads, s); }
        case 20: { const int g = grid_for(blocks_per_sm_x64c<20>(), x64c_paired(20) ? 2 : 1); return launch_x64c<20>(L, g, threads, s); }
        case 21: { const int g = grid_for(blocks_per_sm_x64c<21>(), x64c_paired(21) ? 2 : 1); return launch_x64c<21>(L, g, threads, s); }
        case 22: { const int g = grid_for(blocks_per_sm_x64c<22>(), x64c_paired(22) ? 2 : 1); return launch_x64c<22>(L, g, threads, s); }
        case 23: { const int g = grid_for(blocks_per_sm_x64c<23>(), x64c_paired(23) ? 2 : 1); return launch_x64c<23>(L, g, threads, s); }
        case 24: { const int g = grid_for(blocks_per_sm_x64c<24>(), x64c_paired(24) ? 2 : 1); return launch_x64c<24>(L, g, threads, s); }
        case 25: { const int g = grid_for(blocks_per_sm_x64c<25>(), x64c_paired(25) ? 2 : 1); return launch_x64c<25>(L, g, threads, s); }
        case 26: { const int g = grid_for(blocks_per_sm_x64c<26>(), x64c_paired(26) ? 2 : 1); return launch_x64c<26>(L, g, threads, s); }
        case 27: { const int g = grid_for(blocks_per_sm_x64c<27>(), x64c_paired(27) ? 2 : 1); return launch_x64c<27>(L, g, threads, s); }
        case 28: { const int g = grid_for(blocks_per_sm_x64c<28>(), x64c_paired(28) ? 2 : 1); return launch_x64c<28>(L, g, threads, s); }
        case 29: { const int g = grid_for(blocks_per_sm_x64c<29>(), x64c_paired(29) ? 2 : 1); return launch_x64c<29>(L, g, threads, s); }
        case 30: { const int g = grid_for(blocks_per_sm_x64c<30>(), x64c_paired(30) ? 2 : 1); return launch_x64c<30>(L, g, threads, s); }
        case 31: { const int g = grid_for(blocks_per_sm_x64c<31>(), x64c_paired(31) ? 2 : 1); return launch_x64c<31>(L, g, threads, s); }
        case 32: { const int g = grid_for(blocks_per_sm_x64c<32>(), x64c_paired(32) ? 2 : 1); return launch_x64c<32>(L, g, threads, s); }
        default: return cudaErrorInvalidValue;
    }
}

int dispatch_blocks_per_sm(int kind, int n) {
    // kind: 0 modp, 1 f64, 2 c128, 3 x64 real, 4 x64 complex
    switch (kind) {
        case 0:
            switch (n) {
                case 1: return blocks_per_sm_modp<1>();
                case 2: return blocks_per_sm_modp<2>();
                case 3: return blocks_per_sm_modp<3>();
                case 4: return blocks_per_sm_modp<4>();
                case 5: return blocks_per_sm_modp<5>();
                case 6: return blocks_per_sm_modp<6>();
                case 7: return blocks_per_sm_modp<7>();
                case 8: return blocks_per_sm_modp<8>();
                case 9: return blocks_per_sm_modp<9>();
                case 10: return blocks_per_sm_modp<10>();
                case 11: return blocks_per_sm_modp<11>();
                case 12: return blocks_per_sm_modp<12>();
                case 13: return blocks_per_sm_modp<13>();
                case 14: return blocks_per_sm_modp<14>();
                case 15: return blocks_per_sm_modp<15>();
                case 16: return blocks_per_sm_modp<16>();
                case 17: return blocks_per_sm_modp<17>();
                case 18: return blocks_per_sm_modp<18>();
                case 19: return blocks_per_sm_modp<19>();
                case 20: return blocks_per_sm_modp<20>();
                case 21: return blocks_per_sm_modp<21>();
                case 22: return blocks_per_sm_modp<22>();
                case 23: return blocks_per_sm_modp<23>();
                case 24: return blocks_per_sm_modp<24>();
                case 25: return blocks_per_sm_modp<25>();
                case 26: return blocks_per_sm_modp<26>();
                case 27: return blocks_per_sm_modp<27>();
                case 28: return blocks_per_sm_modp<28>();
                case 29: return blocks_per_sm_modp<29>();
                case 30: return blocks_per_sm_modp<30>();
                case 31: return blocks_per_sm_modp<31>();
                case 32: return blocks_per_sm_modp<32>();
                case 33: return blocks_per_sm_modp<33>();
                case 34: return blocks_per_sm_modp<34>();
                case 35: return blocks_per_sm_modp<35>();
                case 36: return blocks_per_sm_modp<36>();
                case 37: return blocks_per_sm_modp<37>();
                case 38: return blocks_per_sm_modp<38>();
                case 39: return blocks_per_sm_modp<39>();
                case 40: return blocks_per_sm_modp<40>();
                case 41: return blocks_per_sm_modp<41>();
                case 42: return blocks_per_sm_modp<42>();
                case 43: return blocks_per_sm_modp<43>();
                case 44: return blocks_per_sm_modp<44>();
                case 45: return blocks_per_sm_modp<45>();
                case 46: return blocks_per_sm_modp<46>();
                case 47: return blocks_per_sm_modp<47>();
                case 48: return blocks_per_sm_modp<48>();
                default: return 1;
            }
        case 1:
            switch (n) {
                case 1: return blocks_per_sm_f64<1>();
                case 2: return blocks_per_sm_f64<2>();
                case 3: return blocks_per_sm_f64<3>();
                case 4: return blocks_per_sm_f64<4>();
                case 5: return blocks_per_sm_f64<5>();
                case 6: return blocks_per_sm_f64<6>();
                case 7: return blocks_per_sm_f64<7>();
                case 8: return blocks_per_sm_f64<8>();
                case 9: return blocks_per_sm_f64<9>();
                case 10: return blocks_per_sm_f64<10>();
                case 11: return blocks_per_sm_f64<11>();
                case 12: return blocks_per_sm_f64<12>();
                case 13: return blocks_per_sm_f64<13>();
                case 14: return blocks_per_sm_f64<14>();
                case 15: return blocks_per_sm_f64<15>();
                case 16: return blocks_per_sm_f64<16>();
                case 17: return blocks_per_sm_f64<17>();
                case 18: return blocks_per_sm_f64<18>();
                case 19: return blocks_per_sm_f64<19>();
                case 20: return blocks_per_sm_f64<20>();
                case 21: return blocks_per_sm_f64<21>();
                case 22: return blocks_per_sm_f64<22>();
                case 23: return blocks_per_sm_f64<23>();
                case 24: return blocks_per_sm_f64<24>();
                case 25: return blocks_per_sm_f64<25>();
                case 26: return blocks_per_sm_f64<26>();
                case 27: return blocks_per_sm_f64<27>();
                case 28: return blocks_per_sm_f64<28>();
                case 29: return blocks_per_sm_f64<29>();
                case 30: return blocks_per_sm_f64<30>();
                case 31: return blocks_per_sm_f64<31>();
                case 32: return blocks_per_sm_f64<32>();
                default: return 1;
            }
        case 2:
            switch (n) {
                case 1: return blocks_per_sm_c128<1>();
                case 2: return blocks_per_sm_c128<2>();
                case 3: return blocks_per_sm_c128<3>();
                case 4: return blocks_per_sm_c128<4>();
                case 5: return blocks_per_sm_c128<5>();
                case 6: return blocks_per_sm_c128<6>();
                case 7: return blocks_per_sm_c128<7>();
                case 8: return blocks_per_sm_c128<8>();
                case 9: return blocks_per_sm_c128<9>();
                case 10: return blocks_per_sm_c128<10>();
                case 11: return blocks_per_sm_c128<11>();
                case 12: return blocks_per_sm_c128<12>();
                case 13: return blocks_per_sm_c128<13>();
                case 14: return blocks_per_sm_c128<14>();
                case 15: return blocks_per_sm_c128<15>();
                case 16: return blocks_per_sm_c128<16>();
                case 17: return blocks_per_sm_c128<17>();
                case 18: return blocks_per_sm_c128<18>();
                case 19: return blocks_per_sm_c128<19>();
                case 20: return blocks_per_sm_c128<20>();
                case 21: return blocks_per_sm_c128<21>();
                case 22: return blocks_per_sm_c128<22>();
                case 23: return blocks_per_sm_c128<23>();
                case 24: return blocks_per_sm_c128<24>();
                case 25: return blocks_per_sm_c128<25>();
                case 26: return blocks_per_sm_c128<26>();
                case 27: return blocks_per_sm_c128<27>();
                case 28: return blocks_per_sm_c128<28>();
                case 29: return blocks_per_sm_c128<29>();
                case 30: return blocks_per_sm_c128<30>();
                case 31: return blocks_per_sm_c128<31>();
                case 32: return blocks_per_sm_c128<32>();
                default: return 1;
            }
        case 3:
            switch (n) {
                case 1: return blocks_per_sm_x64r<1>();
                case 2: return blocks_per_sm_x64r<2>();
                case 3: return blocks_per_sm_x64r<3>();
                case 4: return blocks_per_sm_x64r<4>();
                case 5: return blocks_per_sm_x64r<5>();
                case 6: return blocks_per_sm_x64r<6>();
                case 7: return blocks_per_sm_x64r<7>();
                case 8: return blocks_per_sm_x64r<8>();
                case 9: return blocks_per_sm_x64r<9>();
                case 10: return blocks_per_sm_x64r<10>();
                case 11: return blocks_per_sm_x64r<11>();
                case 12: return blocks_per_sm_x64r<12>();
                case 13: return blocks_per_sm_x64r<13>();
                case 14: return blocks_per_sm_x64r<14>();
                case 15: return blocks_per_sm_x64r<15>();
                case 16: return blocks_per_sm_x64r<16>();
                case 17: return blocks_per_sm_x64r<17>();
                case 18: return blocks_per_sm_x64r<18>();
                case 19: return blocks_per_sm_x64r<19>();
                case 20: return blocks_per_sm_x64r<20>();
                case 21: return blocks_per_sm_x64r<21>();
                case 22: return blocks_per_sm_x64r<22>();
                case 23: return blocks_per_sm_x64r<23>();
                case 24: return blocks_per_sm_x64r<24>();
                case 25: return blocks_per_sm_x64r<25>();
                case 26: return blocks_per_sm_x64r<26>();
                case 27: return blocks_per_sm_x64r<27>();
                case 28: return blocks_per_sm_x64r<28>();
                case 29: return blocks_per_sm_x64r<29>();
                case 30: return blocks_per_sm_x64r<30>();
                case 31: return blocks_per_sm_x64r<31>();
                case 32: return blocks_per_sm_x64r<32>();
                default: return 1;
            }
        case 4:
            switch (n) {
                case 1: return blocks_per_sm_x64c<1>();
                case 2: return blocks_per_sm_x64c<2>();
                case 3: return blocks_per_sm_x64c<3>();
                case 4: return blocks_per_sm_x64c<4>();
                case 5: return blocks_per_sm_x64c<5>();
                case 6: return blocks_per_sm_x64c<6>();
                case 7: return blocks_per_sm_x64c<7>();
                case 8: return blocks_per_sm_x64c<8>();
                case 9: return blocks_per_sm_x64c<9>();
                case 10: return blocks_per_sm_x64c<10>();
                case 11: return blocks_per_sm_x64c<11>();
                case 12: return blocks_per_sm_x64c<12>();
                case 13: return blocks_per_sm_x64c<13>();
                case 14: return blocks_per_sm_x64c<14>();
                case 15: return blocks_per_sm_x64c<15>();
                case 16: return blocks_per_sm_x64c<16>();
                case 17: return blocks_per_sm_x64c<17>();
                case 18: return blocks_per_sm_x64c<18>();
                case 19: return blocks_per_sm_x64c<19>();
                case 20: return blocks_per_sm_x64c<20>();
                case 21: return blocks_per_sm_x64c<21>();
                case 22: return blocks_per_sm_x64c<22>();
                case 23: return blocks_per_sm_x64c<23>();
                case 24: return blocks_per_sm_x64c<24>();
                case 25: return blocks_per_sm_x64c<25>();
                case 26: return blocks_per_sm_x64c<26>();
                case 27: return blocks_per_sm_x64c<27>();
                case 28: return blocks_per_sm_x64c<28>();
                case 29: return blocks_per_sm_x64c<29>();
                case 30: return blocks_per_sm_x64c<30>();
                case 31: return blocks_per_sm_x64c<31>();
                case 32: return blocks_per_sm_x64c<32>();
                default: return 1;
            }
        default: return 1;
    }
}

}  // namespace permx
