// hierfile.cuh -- binary file of a hierarchy and its boot triplets (host only)
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace samg {

struct HierFile {
    samg_kind kind = SAMG_SVD;
    samg_target target = SAMG_MINIMAL;
    int nb = 0;
    HCsr A;
    std::vector<HCsr> P, Q;               // levels 0 .. n_levels - 2 (Q empty for SPD_EIG)
    std::vector<double> sigma, U, V;      // boot triplets, row-major n_b columns
};

// Throw Error(SAMG_E_INVALID, ...) on an I/O failure or a malformed file
// (wrong magic or version, bad header, truncation, checksum mismatch).  The
// matrices' own structure is checked by the importer.
void write_hierarchy_file(const std::string &path, const HierFile &h);
void read_hierarchy_file(const std::string &path, HierFile &h);

}  // namespace samg
