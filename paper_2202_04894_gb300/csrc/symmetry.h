// The six axis permutations of the hyperoctahedral group (Sec. 4.3), listed
// as sigma arrays (sigma[i] = position of axis i in the canonical offset).
// A transform code is perm_index * 8 + sign_mask (bit i set: axis i negated).
// The host plan encodes codes with this table and the M2L kernel decodes them
// with the same table.
#pragma once

#define DEFMM_PERM_TABLE {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}}
