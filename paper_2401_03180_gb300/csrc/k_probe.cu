// Probe records for the probe-weighted displacement (Sec. II.C, Eq. 17):
// after each step, per replica and species, the summed charge and the summed
// squared displacement |x - x0|^2 of the atoms from their initial positions
// (minimum image of the replica's box).  The weights of Eq. 17 need the whole
// series (their normalisation runs over the probe window), so the series
// stays on the device and is read once.
//
// One thread per atom; block 0 also clears the next record, so a step graph
// needs one launch.  A warp sums its atoms' values per (replica, species)
// key with full-warp butterflies, one distinct key at a time, and one lane
// adds the totals with 64-bit integer atomics.  The squared displacement is
// taken to 2^-40 nm^2 fixed point and split into a high and a low 32-bit
// part, summed in two counters, so the totals are exact and independent of
// the order of the atomics for any atom count below 2^31.
#include "md_internal.cuh"

namespace mdg {
namespace {

__global__ void __launch_bounds__(256) k_probe(Params p)
{
    // a full list stops the step before its forces: the rebuild records it
    if (*p.err & (ERR_CELL | ERR_LIST)) return;
    const long long k = *p.step;                  // record index: steps done
    if (k < 0 || k > p.max_steps) return;         // no slot for it
    if (blockIdx.x == 0 && k < p.max_steps) {        // the next record starts from zero
        for (int t = threadIdx.x; t < p.n_rep * p.n_species; t += blockDim.x) {
            const int r = t / p.n_species, s = t - r * p.n_species;
            long long* rec = p.probe + 3 * (((size_t)r * (p.max_steps + 1) + (size_t)(k + 1)) * p.n_species + s);
            rec[0] = 0; rec[1] = 0; rec[2] = 0;
        }
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < p.n_atoms;
    int key = -1;
    long long vq = 0, vhi = 0, vlo = 0;
    if (valid) {
        const int r = p.rep[i];
        const int s = p.species[i];
        double d[3] = {p.x[i] - p.x0[i], p.y[i] - p.y0[i], p.z[i] - p.z0[i]};
        const Grid& g = p.grid_b[r];
        if (g.periodic)
            for (int c = 0; c < 3; ++c) {
                const int o = beyond_half(d[c], g.box[c]);
                if (o > 0) d[c] -= g.box[c];
                else if (o < 0) d[c] += g.box[c];
            }
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(d2 < 8388607.0)) d2 = 8388607.0;           // below 2^23 nm^2: far beyond any trajectory
        const unsigned long long v = (unsigned long long)__double2ll_rn(d2 * 1099511627776.0);   // 2^40
        vhi = (long long)(v >> 32);
        vlo = (long long)(v & 0xffffffffull);
        vq = p.q[i];
        key = r * p.n_species + s;
    }
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {                                     // warp-uniform loop over distinct keys
        const int src = __ffs(todo) - 1;
        const int k0 = __shfl_sync(0xffffffffu, key, src);
        const bool mine = valid && key == k0;
        long long a = mine ? vq : 0, b = mine ? vhi : 0, c = mine ? vlo : 0;
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == src) {
            const int r = k0 / p.n_species, s = k0 - r * p.n_species;
            long long* rec = p.probe + 3 * (((size_t)r * (p.max_steps + 1) + (size_t)k) * p.n_species + s);
            atomicAdd(reinterpret_cast<unsigned long long*>(rec), (unsigned long long)a);
            atomicAdd(reinterpret_cast<unsigned long long*>(rec + 1), (unsigned long long)b);
            atomicAdd(reinterpret_cast<unsigned long long*>(rec + 2), (unsigned long long)c);
        }
        todo &= ~__ballot_sync(0xffffffffu, mine);
    }
}

// Clears record k of every replica before it is written again (a rebuild
// at an existing step: init, a restored checkpoint, a grown list).
__global__ void k_probe_clear(Params p)
{
    const long long k = *p.step;
    if (k < 0 || k > p.max_steps) return;
    const int n = p.n_rep * p.n_species;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int r = t / p.n_species, s = t - r * p.n_species;
        long long* rec = p.probe + 3 * (((size_t)r * (p.max_steps + 1) + (size_t)k) * p.n_species + s);
        rec[0] = 0; rec[1] = 0; rec[2] = 0;
    }
}

}  // namespace

// rewrite: record k may hold values already (then it is cleared first).
void launch_probe(const Params& p, cudaStream_t s, bool rewrite)
{
    if (!p.probe) return;
    const int nc = p.n_rep * p.n_species;
    if (rewrite) k_probe_clear<<<(nc + 255) / 256, 256, 0, s>>>(p);
    k_probe<<<(p.n_atoms + 255) / 256, 256, 0, s>>>(p);
}

}  // namespace mdg
