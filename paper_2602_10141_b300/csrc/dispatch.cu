// Runtime-n dispatch to the compile-time-n kernels (written by build.py).
#include "common.cuh"

namespace permx {

cudaError_t dispatch_modp(int n, const ModpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    auto grid_for = [&](int bps) {
        uint64_t want = (items + kRyserThreads - 1) / kRyserThreads;
        uint64_t cap = (uint64_t)sm_count() * (uint64_t)bps;
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: return launch_modp<1>(L, grid_for(blocks_per_sm_modp<1>()), s);
        case 2: return launch_modp<2>(L, grid_for(blocks_per_sm_modp<2>()), s);
        case 3: return launch_modp<3>(L, grid_for(blocks_per_sm_modp<3>()), s);
        case 4: return launch_modp<4>(L, grid_for(blocks_per_sm_modp<4>()), s);
        case 5: return launch_modp<5>(L, grid_for(blocks_per_sm_modp<5>()), s);
        case 6: return launch_modp<6>(L, grid_for(blocks_per_sm_modp<6>()), s);
        case 7: return launch_modp<7>(L, grid_for(blocks_per_sm_modp<7>()), s);
        case 8: return launch_modp<8>(L, grid_for(blocks_per_sm_modp<8>()), s);
        case 9: return launch_modp<9>(L, grid_for(blocks_per_sm_modp<9>()), s);
        case 10: return launch_modp<10>(L, grid_for(blocks_per_sm_modp<10>()), s);
        case 11: return launch_modp<11>(L, grid_for(blocks_per_sm_modp<11>()), s);
        case 12: return launch_modp<12>(L, grid_for(blocks_per_sm_modp<12>()), s);
        case 13: return launch_modp<13>(L, grid_for(blocks_per_sm_modp<13>()), s);
        case 14: return launch_modp<14>(L, grid_for(blocks_per_sm_modp<14>()), s);
        case 15: return launch_modp<15>(L, grid_for(blocks_per_sm_modp<15>()), s);
        case 16: return launch_modp<16>(L, grid_for(blocks_per_sm_modp<16>()), s);
        case 17: return launch_modp<17>(L, grid_for(blocks_per_sm_modp<17>()), s);
        case 18: return launch_modp<18>(L, grid_for(blocks_per_sm_modp<18>()), s);
        case 19: return launch_modp<19>(L, grid_for(blocks_per_sm_modp<19>()), s);
        case 20: return launch_modp<20>(L, grid_for(blocks_per_sm_modp<20>()), s);
        case 21: return launch_modp<21>(L, grid_for(blocks_per_sm_modp<21>()), s);
        case 22: return launch_modp<22>(L, grid_for(blocks_per_sm_modp<22>()), s);
        case 23: return launch_modp<23>(L, grid_for(blocks_per_sm_modp<23>()), s);
        case 24: return launch_modp<24>(L, grid_for(blocks_per_sm_modp<24>()), s);
        case 25: return launch_modp<25>(L, grid_for(blocks_per_sm_modp<25>()), s);
        case 26: return launch_modp<26>(L, grid_for(blocks_per_sm_modp<26>()), s);
        case 27: return launch_modp<27>(L, grid_for(blocks_per_sm_modp<27>()), s);
        case 28: return launch_modp<28>(L, grid_for(blocks_per_sm_modp<28>()), s);
        case 29: return launch_modp<29>(L, grid_for(blocks_per_sm_modp<29>()), s);
        case 30: return launch_modp<30>(L, grid_for(blocks_per_sm_modp<30>()), s);
        case 31: return launch_modp<31>(L, grid_for(blocks_per_sm_modp<31>()), s);
        case 32: return launch_modp<32>(L, grid_for(blocks_per_sm_modp<32>()), s);
        case 33: return launch_modp<33>(L, grid_for(blocks_per_sm_modp<33>()), s);
        case 34: return launch_modp<34>(L, grid_for(blocks_per_sm_modp<34>()), s);
        case 35: return launch_modp<35>(L, grid_for(blocks_per_sm_modp<35>()), s);
        case 36: return launch_modp<36>(L, grid_for(blocks_per_sm_modp<36>()), s);
        case 37: return launch_modp<37>(L, grid_for(blocks_per_sm_modp<37>()), s);
        case 38: return launch_modp<38>(L, grid_for(blocks_per_sm_modp<38>()), s);
        case 39: return launch_modp<39>(L, grid_for(blocks_per_sm_modp<39>()), s);
        case 40: return launch_modp<40>(L, grid_for(blocks_per_sm_modp<40>()), s);
        case 41: return launch_modp<41>(L, grid_for(blocks_per_sm_modp<41>()), s);
        case 42: return launch_modp<42>(L, grid_for(blocks_per_sm_modp<42>()), s);
        case 43: return launch_modp<43>(L, grid_for(blocks_per_sm_modp<43>()), s);
        case 44: return launch_modp<44>(L, grid_for(blocks_per_sm_modp<44>()), s);
        case 45: return launch_modp<45>(L, grid_for(blocks_per_sm_modp<45>()), s);
        case 46: return launch_modp<46>(L, grid_for(blocks_per_sm_modp<46>()), s);
        case 47: return launch_modp<47>(L, grid_for(blocks_per_sm_modp<47>()), s);
        case 48: return launch_modp<48>(L, grid_for(blocks_per_sm_modp<48>()), s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_f64(int n, const FpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    auto grid_for = [&](int bps) {
        uint64_t want = (items + kRyserThreads - 1) / kRyserThreads;
        uint64_t cap = (uint64_t)sm_count() * (uint64_t)bps;
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: return launch_f64<1>(L, grid_for(blocks_per_sm_f64<1>()), s);
        case 2: return launch_f64<2>(L, grid_for(blocks_per_sm_f64<2>()), s);
        case 3: return launch_f64<3>(L, grid_for(blocks_per_sm_f64<3>()), s);
        case 4: return launch_f64<4>(L, grid_for(blocks_per_sm_f64<4>()), s);
        case 5: return launch_f64<5>(L, grid_for(blocks_per_sm_f64<5>()), s);
        case 6: return launch_f64<6>(L, grid_for(blocks_per_sm_f64<6>()), s);
        case 7: return launch_f64<7>(L, grid_for(blocks_per_sm_f64<7>()), s);
        case 8: return launch_f64<8>(L, grid_for(blocks_per_sm_f64<8>()), s);
        case 9: return launch_f64<9>(L, grid_for(blocks_per_sm_f64<9>()), s);
        case 10: return launch_f64<10>(L, grid_for(blocks_per_sm_f64<10>()), s);
        case 11: return launch_f64<11>(L, grid_for(blocks_per_sm_f64<11>()), s);
        case 12: return launch_f64<12>(L, grid_for(blocks_per_sm_f64<12>()), s);
        case 13: return launch_f64<13>(L, grid_for(blocks_per_sm_f64<13>()), s);
        case 14: return launch_f64<14>(L, grid_for(blocks_per_sm_f64<14>()), s);
        case 15: return launch_f64<15>(L, grid_for(blocks_per_sm_f64<15>()), s);
        case 16: return launch_f64<16>(L, grid_for(blocks_per_sm_f64<16>()), s);
        case 17: return launch_f64<17>(L, grid_for(blocks_per_sm_f64<17>()), s);
        case 18: return launch_f64<18>(L, grid_for(blocks_per_sm_f64<18>()), s);
        case 19: return launch_f64<19>(L, grid_for(blocks_per_sm_f64<19>()), s);
        case 20: return launch_f64<20>(L, grid_for(blocks_per_sm_f64<20>()), s);
        case 21: return launch_f64<21>(L, grid_for(blocks_per_sm_f64<21>()), s);
        case 22: return launch_f64<22>(L, grid_for(blocks_per_sm_f64<22>()), s);
        case 23: return launch_f64<23>(L, grid_for(blocks_per_sm_f64<23>()), s);
        case 24: return launch_f64<24>(L, grid_for(blocks_per_sm_f64<24>()), s);
        case 25: return launch_f64<25>(L, grid_for(blocks_per_sm_f64<25>()), s);
        case 26: return launch_f64<26>(L, grid_for(blocks_per_sm_f64<26>()), s);
        case 27: return launch_f64<27>(L, grid_for(blocks_per_sm_f64<27>()), s);
        case 28: return launch_f64<28>(L, grid_for(blocks_per_sm_f64<28>()), s);
        case 29: return launch_f64<29>(L, grid_for(blocks_per_sm_f64<29>()), s);
        case 30: return launch_f64<30>(L, grid_for(blocks_per_sm_f64<30>()), s);
        case 31: return launch_f64<31>(L, grid_for(blocks_per_sm_f64<31>()), s);
        case 32: return launch_f64<32>(L, grid_for(blocks_per_sm_f64<32>()), s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_c128(int n, const FpLaunch& L, cudaStream_t s) {
    const uint64_t items = L.item_end - L.item_begin;
    if (items == 0) return cudaSuccess;
    auto grid_for = [&](int bps) {
        uint64_t want = (items + kRyserThreads - 1) / kRyserThreads;
        uint64_t cap = (uint64_t)sm_count() * (uint64_t)bps;
        return (int)(want < cap ? want : cap);
    };
    switch (n) {
        case 1: return launch_c128<1>(L, grid_for(blocks_per_sm_c128<1>()), s);
        case 2: return launch_c128<2>(L, grid_for(blocks_per_sm_c128<2>()), s);
        case 3: return launch_c128<3>(L, grid_for(blocks_per_sm_c128<3>()), s);
        case 4: return launch_c128<4>(L, grid_for(blocks_per_sm_c128<4>()), s);
        case 5: return launch_c128<5>(L, grid_for(blocks_per_sm_c128<5>()), s);
        case 6: return launch_c128<6>(L, grid_for(blocks_per_sm_c128<6>()), s);
        case 7: return launch_c128<7>(L, grid_for(blocks_per_sm_c128<7>()), s);
        case 8: return launch_c128<8>(L, grid_for(blocks_per_sm_c128<8>()), s);
        case 9: return launch_c128<9>(L, grid_for(blocks_per_sm_c128<9>()), s);
        case 10: return launch_c128<10>(L, grid_for(blocks_per_sm_c128<10>()), s);
        case 11: return launch_c128<11>(L, grid_for(blocks_per_sm_c128<11>()), s);
        case 12: return launch_c128<12>(L, grid_for(blocks_per_sm_c128<12>()), s);
        case 13: return launch_c128<13>(L, grid_for(blocks_per_sm_c128<13>()), s);
        case 14: return launch_c128<14>(L, grid_for(blocks_per_sm_c128<14>()), s);
        case 15: return launch_c128<15>(L, grid_for(blocks_per_sm_c128<15>()), s);
        case 16: return launch_c128<16>(L, grid_for(blocks_per_sm_c128<16>()), s);
        case 17: return launch_c128<17>(L, grid_for(blocks_per_sm_c128<17>()), s);
        case 18: return launch_c128<18>(L, grid_for(blocks_per_sm_c128<18>()), s);
        case 19: return launch_c128<19>(L, grid_for(blocks_per_sm_c128<19>()), s);
        case 20: return launch_c128<20>(L, grid_for(blocks_per_sm_c128<20>()), s);
        case 21: return launch_c128<21>(L, grid_for(blocks_per_sm_c128<21>()), s);
        case 22: return launch_c128<22>(L, grid_for(blocks_per_sm_c128<22>()), s);
        case 23: return launch_c128<23>(L, grid_for(blocks_per_sm_c128<23>()), s);
        case 24: return launch_c128<24>(L, grid_for(blocks_per_sm_c128<24>()), s);
        case 25: return launch_c128<25>(L, grid_for(blocks_per_sm_c128<25>()), s);
        case 26: return launch_c128<26>(L, grid_for(blocks_per_sm_c128<26>()), s);
        case 27: return launch_c128<27>(L, grid_for(blocks_per_sm_c128<27>()), s);
        case 28: return launch_c128<28>(L, grid_for(blocks_per_sm_c128<28>()), s);
        case 29: return launch_c128<29>(L, grid_for(blocks_per_sm_c128<29>()), s);
        case 30: return launch_c128<30>(L, grid_for(blocks_per_sm_c128<30>()), s);
        case 31: return launch_c128<31>(L, grid_for(blocks_per_sm_c128<31>()), s);
        case 32: return launch_c128<32>(L, grid_for(blocks_per_sm_c128<32>()), s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace permx
