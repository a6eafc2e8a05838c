// Counter-based random numbers for the device: batch re-draws (am_resample)
// and the CEM sampler.  A draw is a pure function of (seed, stream index,
// draw index), so results do not depend on the launch configuration.
#pragma once

namespace trajam {

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): one output of the generator whose state is x.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform in (0, 1) for draw k of stream l: the top 53 bits of
// SplitMix64(seed XOR SplitMix64(256 l + k)), offset by half a unit.
__device__ __forceinline__ double uniform_draw(unsigned long long seed, unsigned long long l, int k)
{
    const unsigned long long z = splitmix64(seed ^ splitmix64(256ull * l + (unsigned long long)k));
    return (double(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// Standard normal pair from draws 2p, 2p + 1 of stream l (Box-Muller).
__device__ __forceinline__ void normal_pair(unsigned long long seed, unsigned long long l, int p, double &z0,
                                            double &z1)
{
    const double u1 = uniform_draw(seed, l, 2 * p), u2 = uniform_draw(seed, l, 2 * p + 1);
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

}  // namespace trajam
