// Batcher of on-chip launches (onchip.cu), host-only declarations (the serving
// code includes them without the device headers).
#pragma once

// Batched launches (serving): the forward and adjoint launches of several solves of
// one plan shape run as one launch, CTA range b of the grid doing solve b's launch
// with its own tables, buffers and step range.  A host thread bound to a batcher
// (onchip_batcher_bind) hands its on-chip launches to the batcher instead of
// launching them: the batcher waits until every thread that has joined it has handed
// over one launch, then issues them as batched launches on its own stream (ordered
// after each thread's earlier work by events) and makes each thread's stream wait
// for the launch that holds its CTAs.  Each CTA does exactly the arithmetic of the
// unbatched launch, so results do not depend on the batching.
struct OcBatcher;
OcBatcher* onchip_batcher_create(int device);
void onchip_batcher_destroy(OcBatcher* b);
// join: n more threads take part in the next rounds (called before they start, so
// that the first round waits for all of them).  bind: the calling thread, one of
// them, hands its on-chip launches to b.  release: the bound thread has no further
// on-chip launch: it stops taking part (a round waiting only on it launches) and
// unbinds; no-op for an unbound thread.  A bound thread releases before it waits on
// other threads, and every joined thread binds and releases once.
void onchip_batcher_join(OcBatcher* b, int n);
void onchip_batcher_bind(OcBatcher* b);
void onchip_batcher_release();
// Batched launches issued and solves per launch so far.
void onchip_batcher_stats(const OcBatcher* b, long long* launches, long long* members);
