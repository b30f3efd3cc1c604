// Weighted partitioning (Sec. V-C) and the face-local exchange plan.
#pragma once
#include <cstdint>
#include <vector>

#include "host.h"

namespace lts {

struct PartitionStats {
  double max_load = 0, min_load = 0;      // largest / smallest part weight over the mean
  double total_weight = 0;                // element updates per macro step
  double cut_faces = 0;                   // faces whose two elements lie in different parts (per side)
  double msgs_per_macro = 0;              // face-local messages (9 x F values) per macro step
  double buffer_msgs_per_macro = 0;       // whole-buffer messages (9 x B values) the uncompressed scheme sends
};

// part[k] in [0, n_parts) for element weights 2^(N_c-1-cluster); see host_partition.cpp.
void partition_elements(const Mesh& m, const std::vector<int32_t>& cluster, int nc, int n_parts,
                        std::vector<int32_t>& part, PartitionStats* stats);

// One receiver-side face whose neighbour lies in another part: the sender computes
// H = X F-_{send_face, orient} from its buffer X and sends it; the receiver applies the
// flux and F^ of recv_face.
struct CutFace {
  int64_t recv_elem, send_elem;
  int32_t recv_face, send_face, orient, recv_part, send_part, recv_cluster;
};

// Every cut face, in message order: by (receiving part, sending part), then receiver
// cluster, element and face.
void cut_faces(const Mesh& m, const std::vector<int32_t>& part, const std::vector<int32_t>& cluster,
               std::vector<CutFace>& out);

}  // namespace lts
