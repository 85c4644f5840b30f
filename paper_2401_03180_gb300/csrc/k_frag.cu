// Fragments and their ion yields (Sec. III: fractional ion yields by mass and
// charge).  The union-find links come from the pair-list walk (FragOp in
// k_pair.cu); this file holds the per-atom passes around it: initialise the
// parents, resolve every atom's root (its fragment's smallest atom index),
// sum the fragments' mass numbers and charges at their roots, and count the
// fragments per replica by (mass number, charge).
#include <algorithm>

#include "md_internal.cuh"

namespace mdg {
namespace {

struct MassNumbers {
    int a[kMaxSpecies];
};

__global__ void k_frag_init(int n, int* parent, int* mass, int* charge)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        parent[i] = i;
        mass[i] = 0;
        charge[i] = 0;
    }
}

// Root of every atom (parents only decrease, so the walk ends), then the
// atom's mass number and charge added at the root.
__global__ void k_frag_root(Params p, const int* parent, int* label, int* mass, int* charge, MassNumbers an)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n_atoms; i += gridDim.x * blockDim.x) {
        int x = i;
        for (int it = 0; it < p.n_atoms; ++it) {       // at most i steps: each one decreases x
            const int px = __ldcg(parent + x);
            if (px == x) break;
            x = px;
        }
        label[i] = x;
        atomicAdd(mass + x, an.a[p.species[i]]);
        atomicAdd(charge + x, (int)p.q[i]);
    }
}

__global__ void k_frag_count(Params p, const int* label, const int* mass, const int* charge, int mass_max,
                             int charge_max, unsigned long long* counts)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n_atoms; i += gridDim.x * blockDim.x) {
        if (label[i] != i) continue;
        const int m = min(mass[i], mass_max), z = min(charge[i], charge_max);
        atomicAdd(counts + ((size_t)p.rep[i] * (mass_max + 1) + m) * (charge_max + 1) + z, 1ull);
    }
}

}  // namespace

void launch_frag_init(const Params& p, cudaStream_t s, int* parent, int* mass, int* charge)
{
    const int blocks = std::max(1, std::min((p.n_atoms + 255) / 256, 4096));
    k_frag_init<<<blocks, 256, 0, s>>>(p.n_atoms, parent, mass, charge);
}

void launch_frag_count(const Params& p, cudaStream_t s, const int* parent, int* label, int* mass, int* charge,
                       const int* mass_number, int mass_max, int charge_max, unsigned long long* counts)
{
    MassNumbers an{};
    for (int k = 0; k < p.n_species && k < kMaxSpecies; ++k) an.a[k] = mass_number[k];
    const int blocks = std::max(1, std::min((p.n_atoms + 255) / 256, 4096));
    k_frag_root<<<blocks, 256, 0, s>>>(p, parent, label, mass, charge, an);
    k_frag_count<<<blocks, 256, 0, s>>>(p, label, mass, charge, mass_max, charge_max, counts);
}

}  // namespace mdg
