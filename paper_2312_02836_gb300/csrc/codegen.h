// codegen.h -- network-specialised kernel: source generation and run-time
// compilation (codegen.cpp).  Host-only; not part of the ABI.
#pragma once
#include <string>
#include <vector>

#include "blob.h"

namespace nb {

// Storage variant 1..3 for `variant`, 0 = chosen from the network's sizes.
int resolve_variant(const BlobHeader& h, int variant);

// Whether the automatic choice specialises this network (its straight-line
// code stays small enough to compile in seconds).
bool specialize_auto_ok(const BlobHeader& h);

// CUDA source of the specialised kernel `nb_spec_burn` for a compiled network.
std::string specialized_source(const std::vector<uint8_t>& blob, int variant);

// Compile to an sm_103a cubin with the run-time compiler (loaded on first
// use).  NB_OK or NB_E_COMPILE; *log receives the compiler's log.
int compile_specialized(const std::string& src, std::vector<char>* cubin,
                        std::string* log, bool verbose);

}  // namespace nb
