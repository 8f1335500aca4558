// Generated by gen_twiddles_hi.py: W_n^m = exp(-2 pi i m/n) as double pairs
// {cos_hi, cos_lo, sin_hi, sin_lo}, hi + lo accurate to ~2^-106.
#pragma once
static const double kTw64Hi[64][4] = {
    {0x1.0000000000000p+0, 0x0.0p+0, 0x0.0p+0, 0x0.0p+0},
    {0x1.fd88da3d12526p-1, -0x1.87df6378811c7p-55, -0x1.917a6bc29b42cp-4, 0x1.e2718d26ed688p-60},
    {0x1.f6297cff75cb0p-1, 0x1.562172a361fd3p-56, -0x1.8f8b83c69a60bp-3, 0x1.26d19b9ff8d82p-57},
    {0x1.e9f4156c62ddap-1, 0x1.760b1e2e3f81ep-55, -0x1.294062ed59f06p-2, 0x1.5d28da2c4612dp-56},
    {0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56, -0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57},
    {0x1.c38b2f180bdb1p-1, -0x1.6e0b1757c8d07p-56, -0x1.e2b5d3806f63bp-2, -0x1.e0d891d3c6841p-58},
    {0x1.a9b66290ea1a3p-1, 0x1.9f630e8b6dac8p-60, -0x1.1c73b39ae68c8p-1, -0x1.b25dd267f6600p-55},
    {0x1.8bc806b151741p-1, -0x1.2c5e12ed1336dp-55, -0x1.44cf325091dd6p-1, -0x1.8076a2cfdc6b3p-57},
    {0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55, -0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55},
    {0x1.44cf325091dd6p-1, 0x1.8076a2cfdc6b3p-57, -0x1.8bc806b151741p-1, 0x1.2c5e12ed1336dp-55},
    {0x1.1c73b39ae68c8p-1, 0x1.b25dd267f6600p-55, -0x1.a9b66290ea1a3p-1, -0x1.9f630e8b6dac8p-60},
    {0x1.e2b5d3806f63bp-2, 0x1.e0d891d3c6841p-58, -0x1.c38b2f180bdb1p-1, 0x1.6e0b1757c8d07p-56},
    {0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57, -0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56},
    {0x1.294062ed59f06p-2, -0x1.5d28da2c4612dp-56, -0x1.e9f4156c62ddap-1, -0x1.760b1e2e3f81ep-55},
    {0x1.8f8b83c69a60bp-3, -0x1.26d19b9ff8d82p-57, -0x1.f6297cff75cb0p-1, -0x1.562172a361fd3p-56},
    {0x1.917a6bc29b42cp-4, -0x1.e2718d26ed688p-60, -0x1.fd88da3d12526p-1, 0x1.87df6378811c7p-55},
    {0x0.0p+0, 0x0.0p+0, -0x1.0000000000000p+0, 0x0.0p+0},
    {-0x1.917a6bc29b42cp-4, 0x1.e2718d26ed688p-60, -0x1.fd88da3d12526p-1, 0x1.87df6378811c7p-55},
    {-0x1.8f8b83c69a60bp-3, 0x1.26d19b9ff8d82p-57, -0x1.f6297cff75cb0p-1, -0x1.562172a361fd3p-56},
    {-0x1.294062ed59f06p-2, 0x1.5d28da2c4612dp-56, -0x1.e9f4156c62ddap-1, -0x1.760b1e2e3f81ep-55},
    {-0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57, -0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56},
    {-0x1.e2b5d3806f63bp-2, -0x1.e0d891d3c6841p-58, -0x1.c38b2f180bdb1p-1, 0x1.6e0b1757c8d07p-56},
    {-0x1.1c73b39ae68c8p-1, -0x1.b25dd267f6600p-55, -0x1.a9b66290ea1a3p-1, -0x1.9f630e8b6dac8p-60},
    {-0x1.44cf325091dd6p-1, -0x1.8076a2cfdc6b3p-57, -0x1.8bc806b151741p-1, 0x1.2c5e12ed1336dp-55},
    {-0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55, -0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55},
    {-0x1.8bc806b151741p-1, 0x1.2c5e12ed1336dp-55, -0x1.44cf325091dd6p-1, -0x1.8076a2cfdc6b3p-57},
    {-0x1.a9b66290ea1a3p-1, -0x1.9f630e8b6dac8p-60, -0x1.1c73b39ae68c8p-1, -0x1.b25dd267f6600p-55},
    {-0x1.c38b2f180bdb1p-1, 0x1.6e0b1757c8d07p-56, -0x1.e2b5d3806f63bp-2, -0x1.e0d891d3c6841p-58},
    {-0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56, -0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57},
    {-0x1.e9f4156c62ddap-1, -0x1.760b1e2e3f81ep-55, -0x1.294062ed59f06p-2, 0x1.5d28da2c4612dp-56},
    {-0x1.f6297cff75cb0p-1, -0x1.562172a361fd3p-56, -0x1.8f8b83c69a60bp-3, 0x1.26d19b9ff8d82p-57},
    {-0x1.fd88da3d12526p-1, 0x1.87df6378811c7p-55, -0x1.917a6bc29b42cp-4, 0x1.e2718d26ed688p-60},
    {-0x1.0000000000000p+0, 0x0.0p+0, -0x0.0p+0, 0x0.0p+0},
    {-0x1.fd88da3d12526p-1, 0x1.87df6378811c7p-55, 0x1.917a6bc29b42cp-4, -0x1.e2718d26ed688p-60},
    {-0x1.f6297cff75cb0p-1, -0x1.562172a361fd3p-56, 0x1.8f8b83c69a60bp-3, -0x1.26d19b9ff8d82p-57},
    {-0x1.e9f4156c62ddap-1, -0x1.760b1e2e3f81ep-55, 0x1.294062ed59f06p-2, -0x1.5d28da2c4612dp-56},
    {-0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56, 0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57},
    {-0x1.c38b2f180bdb1p-1, 0x1.6e0b1757c8d07p-56, 0x1.e2b5d3806f63bp-2, 0x1.e0d891d3c6841p-58},
    {-0x1.a9b66290ea1a3p-1, -0x1.9f630e8b6dac8p-60, 0x1.1c73b39ae68c8p-1, 0x1.b25dd267f6600p-55},
    {-0x1.8bc806b151741p-1, 0x1.2c5e12ed1336dp-55, 0x1.44cf325091dd6p-1, 0x1.8076a2cfdc6b3p-57},
    {-0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55, 0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55},
    {-0x1.44cf325091dd6p-1, -0x1.8076a2cfdc6b3p-57, 0x1.8bc806b151741p-1, -0x1.2c5e12ed1336dp-55},
    {-0x1.1c73b39ae68c8p-1, -0x1.b25dd267f6600p-55, 0x1.a9b66290ea1a3p-1, 0x1.9f630e8b6dac8p-60},
    {-0x1.e2b5d3806f63bp-2, -0x1.e0d891d3c6841p-58, 0x1.c38b2f180bdb1p-1, -0x1.6e0b1757c8d07p-56},
    {-0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57, 0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56},
    {-0x1.294062ed59f06p-2, 0x1.5d28da2c4612dp-56, 0x1.e9f4156c62ddap-1, 0x1.760b1e2e3f81ep-55},
    {-0x1.8f8b83c69a60bp-3, 0x1.26d19b9ff8d82p-57, 0x1.f6297cff75cb0p-1, 0x1.562172a361fd3p-56},
    {-0x1.917a6bc29b42cp-4, 0x1.e2718d26ed688p-60, 0x1.fd88da3d12526p-1, -0x1.87df6378811c7p-55},
    {-0x0.0p+0, 0x0.0p+0, 0x1.0000000000000p+0, 0x0.0p+0},
    {0x1.917a6bc29b42cp-4, -0x1.e2718d26ed688p-60, 0x1.fd88da3d12526p-1, -0x1.87df6378811c7p-55},
    {0x1.8f8b83c69a60bp-3, -0x1.26d19b9ff8d82p-57, 0x1.f6297cff75cb0p-1, 0x1.562172a361fd3p-56},
    {0x1.294062ed59f06p-2, -0x1.5d28da2c4612dp-56, 0x1.e9f4156c62ddap-1, 0x1.760b1e2e3f81ep-55},
    {0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57, 0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56},
    {0x1.e2b5d3806f63bp-2, 0x1.e0d891d3c6841p-58, 0x1.c38b2f180bdb1p-1, -0x1.6e0b1757c8d07p-56},
    {0x1.1c73b39ae68c8p-1, 0x1.b25dd267f6600p-55, 0x1.a9b66290ea1a3p-1, 0x1.9f630e8b6dac8p-60},
    {0x1.44cf325091dd6p-1, 0x1.8076a2cfdc6b3p-57, 0x1.8bc806b151741p-1, -0x1.2c5e12ed1336dp-55},
    {0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55, 0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55},
    {0x1.8bc806b151741p-1, -0x1.2c5e12ed1336dp-55, 0x1.44cf325091dd6p-1, 0x1.8076a2cfdc6b3p-57},
    {0x1.a9b66290ea1a3p-1, 0x1.9f630e8b6dac8p-60, 0x1.1c73b39ae68c8p-1, 0x1.b25dd267f6600p-55},
    {0x1.c38b2f180bdb1p-1, -0x1.6e0b1757c8d07p-56, 0x1.e2b5d3806f63bp-2, 0x1.e0d891d3c6841p-58},
    {0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56, 0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57},
    {0x1.e9f4156c62ddap-1, 0x1.760b1e2e3f81ep-55, 0x1.294062ed59f06p-2, -0x1.5d28da2c4612dp-56},
    {0x1.f6297cff75cb0p-1, 0x1.562172a361fd3p-56, 0x1.8f8b83c69a60bp-3, -0x1.26d19b9ff8d82p-57},
    {0x1.fd88da3d12526p-1, -0x1.87df6378811c7p-55, 0x1.917a6bc29b42cp-4, -0x1.e2718d26ed688p-60},
};
static const double kTw48Hi[48][4] = {
    {0x1.0000000000000p+0, 0x0.0p+0, 0x0.0p+0, 0x0.0p+0},
    {0x1.fb9ea92ec689bp-1, 0x1.0b62768cd6744p-55, -0x1.0b5150f6da2d1p-3, 0x1.6275d70b88e44p-57},
    {0x1.ee8dd4748bf15p-1, -0x1.d5ba34b10d383p-56, -0x1.0907dc1930690p-2, -0x1.a5ec4dc53f528p-56},
    {0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56, -0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57},
    {0x1.bb67ae8584caap-1, 0x1.cec95d0b5c1e3p-55, -0x1.0000000000000p-1, 0x0.0p+0},
    {0x1.963268b572492p-1, -0x1.28d66f013c37ep-61, -0x1.37af93f9513eap-1, 0x1.2fd3a447a5e70p-56},
    {0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55, -0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55},
    {0x1.37af93f9513eap-1, -0x1.2fd3a447a5e70p-56, -0x1.963268b572492p-1, 0x1.28d66f013c37ep-61},
    {0x1.0000000000000p-1, 0x0.0p+0, -0x1.bb67ae8584caap-1, -0x1.cec95d0b5c1e3p-55},
    {0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57, -0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56},
    {0x1.0907dc1930690p-2, 0x1.a5ec4dc53f528p-56, -0x1.ee8dd4748bf15p-1, 0x1.d5ba34b10d383p-56},
    {0x1.0b5150f6da2d1p-3, -0x1.6275d70b88e44p-57, -0x1.fb9ea92ec689bp-1, -0x1.0b62768cd6744p-55},
    {0x0.0p+0, 0x0.0p+0, -0x1.0000000000000p+0, 0x0.0p+0},
    {-0x1.0b5150f6da2d1p-3, 0x1.6275d70b88e44p-57, -0x1.fb9ea92ec689bp-1, -0x1.0b62768cd6744p-55},
    {-0x1.0907dc1930690p-2, -0x1.a5ec4dc53f528p-56, -0x1.ee8dd4748bf15p-1, 0x1.d5ba34b10d383p-56},
    {-0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57, -0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56},
    {-0x1.0000000000000p-1, 0x0.0p+0, -0x1.bb67ae8584caap-1, -0x1.cec95d0b5c1e3p-55},
    {-0x1.37af93f9513eap-1, 0x1.2fd3a447a5e70p-56, -0x1.963268b572492p-1, 0x1.28d66f013c37ep-61},
    {-0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55, -0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55},
    {-0x1.963268b572492p-1, 0x1.28d66f013c37ep-61, -0x1.37af93f9513eap-1, 0x1.2fd3a447a5e70p-56},
    {-0x1.bb67ae8584caap-1, -0x1.cec95d0b5c1e3p-55, -0x1.0000000000000p-1, 0x0.0p+0},
    {-0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56, -0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57},
    {-0x1.ee8dd4748bf15p-1, 0x1.d5ba34b10d383p-56, -0x1.0907dc1930690p-2, -0x1.a5ec4dc53f528p-56},
    {-0x1.fb9ea92ec689bp-1, -0x1.0b62768cd6744p-55, -0x1.0b5150f6da2d1p-3, 0x1.6275d70b88e44p-57},
    {-0x1.0000000000000p+0, 0x0.0p+0, -0x0.0p+0, 0x0.0p+0},
    {-0x1.fb9ea92ec689bp-1, -0x1.0b62768cd6744p-55, 0x1.0b5150f6da2d1p-3, -0x1.6275d70b88e44p-57},
    {-0x1.ee8dd4748bf15p-1, 0x1.d5ba34b10d383p-56, 0x1.0907dc1930690p-2, 0x1.a5ec4dc53f528p-56},
    {-0x1.d906bcf328d46p-1, -0x1.457e610231ac2p-56, 0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57},
    {-0x1.bb67ae8584caap-1, -0x1.cec95d0b5c1e3p-55, 0x1.0000000000000p-1, 0x0.0p+0},
    {-0x1.963268b572492p-1, 0x1.28d66f013c37ep-61, 0x1.37af93f9513eap-1, -0x1.2fd3a447a5e70p-56},
    {-0x1.6a09e667f3bcdp-1, 0x1.bdd3413b26456p-55, 0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55},
    {-0x1.37af93f9513eap-1, 0x1.2fd3a447a5e70p-56, 0x1.963268b572492p-1, -0x1.28d66f013c37ep-61},
    {-0x1.0000000000000p-1, 0x0.0p+0, 0x1.bb67ae8584caap-1, 0x1.cec95d0b5c1e3p-55},
    {-0x1.87de2a6aea963p-2, 0x1.72cedd3d5a610p-57, 0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56},
    {-0x1.0907dc1930690p-2, -0x1.a5ec4dc53f528p-56, 0x1.ee8dd4748bf15p-1, -0x1.d5ba34b10d383p-56},
    {-0x1.0b5150f6da2d1p-3, 0x1.6275d70b88e44p-57, 0x1.fb9ea92ec689bp-1, 0x1.0b62768cd6744p-55},
    {-0x0.0p+0, 0x0.0p+0, 0x1.0000000000000p+0, 0x0.0p+0},
    {0x1.0b5150f6da2d1p-3, -0x1.6275d70b88e44p-57, 0x1.fb9ea92ec689bp-1, 0x1.0b62768cd6744p-55},
    {0x1.0907dc1930690p-2, 0x1.a5ec4dc53f528p-56, 0x1.ee8dd4748bf15p-1, -0x1.d5ba34b10d383p-56},
    {0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57, 0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56},
    {0x1.0000000000000p-1, 0x0.0p+0, 0x1.bb67ae8584caap-1, 0x1.cec95d0b5c1e3p-55},
    {0x1.37af93f9513eap-1, -0x1.2fd3a447a5e70p-56, 0x1.963268b572492p-1, -0x1.28d66f013c37ep-61},
    {0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55, 0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55},
    {0x1.963268b572492p-1, -0x1.28d66f013c37ep-61, 0x1.37af93f9513eap-1, -0x1.2fd3a447a5e70p-56},
    {0x1.bb67ae8584caap-1, 0x1.cec95d0b5c1e3p-55, 0x1.0000000000000p-1, 0x0.0p+0},
    {0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56, 0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57},
    {0x1.ee8dd4748bf15p-1, -0x1.d5ba34b10d383p-56, 0x1.0907dc1930690p-2, 0x1.a5ec4dc53f528p-56},
    {0x1.fb9ea92ec689bp-1, 0x1.0b62768cd6744p-55, 0x1.0b5150f6da2d1p-3, -0x1.6275d70b88e44p-57},
};
#ifndef LBO_HD
#ifdef __CUDACC__
#define LBO_HD __host__ __device__
#else
#define LBO_HD
#endif
#endif
// W_32^m, m < 16: kind 0: sc (1 + i q); kind 1: sc (q + i)
struct ScaledTw {
  int kind;
  double sc, q;
};
LBO_HD constexpr ScaledTw scaled_tw32(int m) {
  switch (m) {
    case 0: return {0, 0x1.0000000000000p+0, 0x0.0p+0};
    case 1: return {0, 0x1.f6297cff75cb0p-1, -0x1.975f5e0553158p-3};
    case 2: return {0, 0x1.d906bcf328d46p-1, -0x1.a827999fcef32p-2};
    case 3: return {0, 0x1.a9b66290ea1a3p-1, -0x1.561b82ab7f990p-1};
    case 4: return {0, 0x1.6a09e667f3bcdp-1, -0x1.0000000000000p+0};
    case 5: return {1, -0x1.a9b66290ea1a3p-1, -0x1.561b82ab7f990p-1};
    case 6: return {1, -0x1.d906bcf328d46p-1, -0x1.a827999fcef32p-2};
    case 7: return {1, -0x1.f6297cff75cb0p-1, -0x1.975f5e0553158p-3};
    case 8: return {1, -0x1.0000000000000p+0, -0x0.0p+0};
    case 9: return {1, -0x1.f6297cff75cb0p-1, 0x1.975f5e0553158p-3};
    case 10: return {1, -0x1.d906bcf328d46p-1, 0x1.a827999fcef32p-2};
    case 11: return {1, -0x1.a9b66290ea1a3p-1, 0x1.561b82ab7f990p-1};
    case 12: return {0, -0x1.6a09e667f3bcdp-1, 0x1.0000000000000p+0};
    case 13: return {0, -0x1.a9b66290ea1a3p-1, 0x1.561b82ab7f990p-1};
    case 14: return {0, -0x1.d906bcf328d46p-1, 0x1.a827999fcef32p-2};
    case 15: return {0, -0x1.f6297cff75cb0p-1, 0x1.975f5e0553158p-3};
    default: return {0, 0.0, 0.0};
  }
}
// cos(2 pi m / 32), m < 32, correctly rounded
LBO_HD constexpr double cos32(int m) {
  switch (m) {
    case 0: return 0x1.0000000000000p+0;
    case 1: return 0x1.f6297cff75cb0p-1;
    case 2: return 0x1.d906bcf328d46p-1;
    case 3: return 0x1.a9b66290ea1a3p-1;
    case 4: return 0x1.6a09e667f3bcdp-1;
    case 5: return 0x1.1c73b39ae68c8p-1;
    case 6: return 0x1.87de2a6aea963p-2;
    case 7: return 0x1.8f8b83c69a60bp-3;
    case 8: return 0x0.0p+0;
    case 9: return -0x1.8f8b83c69a60bp-3;
    case 10: return -0x1.87de2a6aea963p-2;
    case 11: return -0x1.1c73b39ae68c8p-1;
    case 12: return -0x1.6a09e667f3bcdp-1;
    case 13: return -0x1.a9b66290ea1a3p-1;
    case 14: return -0x1.d906bcf328d46p-1;
    case 15: return -0x1.f6297cff75cb0p-1;
    case 16: return -0x1.0000000000000p+0;
    case 17: return -0x1.f6297cff75cb0p-1;
    case 18: return -0x1.d906bcf328d46p-1;
    case 19: return -0x1.a9b66290ea1a3p-1;
    case 20: return -0x1.6a09e667f3bcdp-1;
    case 21: return -0x1.1c73b39ae68c8p-1;
    case 22: return -0x1.87de2a6aea963p-2;
    case 23: return -0x1.8f8b83c69a60bp-3;
    case 24: return -0x0.0p+0;
    case 25: return 0x1.8f8b83c69a60bp-3;
    case 26: return 0x1.87de2a6aea963p-2;
    case 27: return 0x1.1c73b39ae68c8p-1;
    case 28: return 0x1.6a09e667f3bcdp-1;
    case 29: return 0x1.a9b66290ea1a3p-1;
    case 30: return 0x1.d906bcf328d46p-1;
    case 31: return 0x1.f6297cff75cb0p-1;
    default: return 0.0;
  }
}
