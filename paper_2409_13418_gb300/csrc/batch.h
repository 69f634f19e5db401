// batch.h -- network evaluations shared by several contexts (a batch group).
//
// Contexts that join a group evaluate the network queries of their search
// stages (the 1D bisection and the 2D face search, Sec. 5.1 and 5.2: one
// evaluation per search step over all active elements) together: each call
// waits until every context currently inside a search stage has made one,
// then one thread merges their query lists on the group's stream, runs the
// tiered evaluation once over all of them, and returns every logit to its
// caller's buffer, stream ordered.  Latent-conditioned shapes of one network
// differ only in their folded first-layer bias, which each query carries as
// a row of the group's bias table.  Every row of a network launch is
// computed independently of the others, so each shape's logits, decisions
// and mesh are those of its extraction alone.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/odc.h"

namespace odc {

struct MlpState;
struct BatchGroup;

odc_status batch_create(int device, BatchGroup** out, std::string* err);
void batch_destroy(BatchGroup* g);
// Statistics: merged evaluation rounds and member calls they served.
void batch_stats(const BatchGroup* g, int64_t* rounds, int64_t* calls);

// Bind a context's network state to group g (NULL: unbind).  m is the MLP
// source just uploaded to st (NULL for a resident source: the binding made
// at its upload stays).  The first bound source sets the group's network; a
// state whose network (B, W, b) or precision differs from it evaluates on
// its own.
odc_status batch_bind(MlpState* st, BatchGroup* g, const odc_mlp* m, std::string* err);
void batch_unbind(MlpState* st);

// Search-stage brackets (members only; no-ops otherwise).
void batch_enter(MlpState* st);
odc_status batch_leave(MlpState* st, std::string* err);
bool batch_active(const MlpState* st);

// One shared evaluation call: the logits of n queries (n_dev: device count,
// at most n_max; else n_max) at pts into z, with optional routing hints,
// stream ordered on s.
odc_status batch_eval(MlpState* st, const float3* pts, int64_t n_max, const unsigned long long* n_dev, float* z,
                      const float* hint, cudaStream_t s, std::string* err);

}  // namespace odc
