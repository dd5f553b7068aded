"""FP64 CPU oracle of FARM relational retrieval.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package.  The product path (the CUDA library and
its binding) never does.
"""
from .oracle import (ABOVE, BELOW, LEFT_OF, RIGHT_OF, NEAR, NEXT_TO, ON, IN_FRONT_OF, BEHIND,
                     CLOSEST, FARTHEST, NEAR_H, INSIDE, BETWEEN, BETWEEN_AND, OracleParams, build, load, cosines, ranks, relation,
                     relation_in, sigmoid, query_all, query_bounds, batch, topk, num_threads,
                     query_mc, query_bounds_mc, between, hellinger, associate)

__all__ = ["ABOVE", "BELOW", "LEFT_OF", "RIGHT_OF", "NEAR", "NEXT_TO", "ON", "IN_FRONT_OF", "BEHIND",
           "CLOSEST", "FARTHEST", "NEAR_H", "INSIDE", "BETWEEN", "BETWEEN_AND", "OracleParams", "build", "load", "cosines", "ranks", "relation",
           "relation_in", "sigmoid", "query_all", "query_bounds", "batch", "topk", "num_threads",
           "query_mc", "query_bounds_mc", "between", "hellinger", "associate"]
