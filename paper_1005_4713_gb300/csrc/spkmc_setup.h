// spkmc_setup.h -- host-side launchers of the set-up kernels that work on a
// range of domain layers, so that writing the spins can overlap the refresh
// of the layers already written with the transfer of the next ones.
#pragma once

#include "spkmc_internal.h"

namespace spkmc {

// Whether the tiled transposition takes host-order spins at src (packed: one
// bit per site, else int8) for this lattice.
bool pack_is_tiled(const LatticeDesc &d, const void *src, bool packed);
// The tiled pack of domain layers dz in [z0, z1) only, on at most cap CTAs
// (EINVAL where the tiled pack does not apply or the range is empty).
int launch_pack_layers(const LatticeDesc &d, const void *src, bool packed, int z0, int z1, int cap, void *stream);
// Ghost faces, class counts and (with MB) M and B of the domains of layers
// dz in [z0, z1), in one pass; the rows of layers z0 - 1 .. z1 (periodic)
// must be in place.
int launch_refresh_layers(const LatticeDesc &d, long long *MB, int z0, int z1, void *stream);

} // namespace spkmc
