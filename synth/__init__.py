"""Seeded synthetic scenes and queries shared by the FP64 oracle and the CUDA path.

This package draws random numbers and lays them out; it holds none of the
retrieval method's arithmetic (no cosines, ranks, predicates or scores).
"""
from .scenes import (Scene, QueryBatch, make_scene, make_queries, workload,
                     WORKLOADS, Spaces, add_spaces, ChannelQueries, channel_queries, PAPER_CHANNELS,
                     make_association)

__all__ = ["Scene", "QueryBatch", "make_scene", "make_queries", "workload",
           "WORKLOADS", "Spaces", "add_spaces", "ChannelQueries", "channel_queries", "PAPER_CHANNELS",
           "make_association"]
