// Oracle: counter-based generator and object-state hash. Test infrastructure only.
//
// The applications draw their random choices from a counter-based generator
// keyed on (seed, stream, step, cell), so that a result does not depend on
// which thread or in which order a choice is made. The generator is
// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): state advances by the golden-ratio increment
// and each output is the state passed through the 64-bit finalizer.
//
//   splitmix_at(s, n) = mix64(s + (n + 1) * GAMMA)    -- n-th output from seed s
//   rand(seed, stream, step, cell) =
//       splitmix_at(splitmix_at(splitmix_at(seed, stream), step), cell)
//
// Object-state hash: an object of type t with 32-bit field words w_0..w_{k-1}
// hashes to
//   h_0 = mix64(t + GAMMA);  h_{i+1} = mix64((h_i ^ w_i) + GAMMA);  h = h_k
// and the state hash of a set of objects is the sum of their h modulo 2^64,
// which does not depend on where or in what order the objects are stored.
#include "oracle.h"

namespace {
constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
}

extern "C" uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" uint64_t orc_splitmix_at(uint64_t s, uint64_t n) {
    return orc_mix64(s + (n + 1) * GAMMA);
}

extern "C" uint64_t orc_rand(uint64_t seed, uint64_t stream, uint64_t step, uint64_t cell) {
    uint64_t k = orc_splitmix_at(seed, stream);
    k = orc_splitmix_at(k, step);
    return orc_splitmix_at(k, cell);
}

extern "C" uint64_t orc_obj_hash(uint32_t type_id, const uint32_t* words, int n_words) {
    uint64_t h = orc_mix64((uint64_t)type_id + GAMMA);
    for (int i = 0; i < n_words; ++i) h = orc_mix64((h ^ (uint64_t)words[i]) + GAMMA);
    return h;
}
