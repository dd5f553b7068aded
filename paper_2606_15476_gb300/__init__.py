"""GB300-native (sm_103a) relational retrieval over an object-level spatial memory.

The compute path is the CUDA library libfarm.so (C ABI in include/farm.h);
`farm` is its thin ctypes binding with the same entry-point names.
"""
from . import farm
from .farm import (FarmError, FarmParams, farm_candidates, farm_create, farm_default_params,
                   farm_destroy, farm_last_error, farm_memory_upload, farm_memory_release, farm_query_batch,
                   farm_rank_rows_noalloc, farm_mlp_set, farm_mlp_get, farm_mlp_loss_grad,
                   farm_mlp_train, farm_mlp_embed, PREC_LEARNED,
                   farm_scene_info, farm_select_fallbacks, farm_sim_tuning, farm_sim_variant_pin, farm_similarity_variant, farm_set_profiling, farm_similarity, farm_stage_times, farm_sync, farm_topk,
                   farm_version, farm_memory_add_space, farm_query_batch_rrf, FarmChannel, farm_associate, GRAPH, UNFUSED, PREC_FP32, PREC_BF16, PREC_FP8, PREC_FP32_SIMT, PTR_DEVICE)

__all__ = ["farm", "FarmError", "FarmParams", "farm_candidates", "farm_create",
           "farm_default_params", "farm_destroy", "farm_last_error", "farm_memory_upload", "farm_memory_release",
           "farm_query_batch", "farm_rank_rows_noalloc", "farm_mlp_set", "farm_mlp_get",
           "farm_mlp_loss_grad", "farm_mlp_train", "farm_mlp_embed", "PREC_LEARNED", "farm_scene_info", "farm_select_fallbacks", "farm_sim_tuning", "farm_sim_variant_pin", "farm_similarity_variant", "farm_set_profiling", "farm_similarity", "farm_stage_times",
           "farm_sync", "farm_topk", "farm_version", "PREC_FP32", "PREC_BF16", "PREC_FP8", "PREC_FP32_SIMT",
           "PTR_DEVICE", "GRAPH", "UNFUSED", "farm_memory_add_space", "farm_query_batch_rrf", "FarmChannel", "farm_associate"]
