"""GB300 (sm_103a) sort-based grouping with early aggregation and wide merging.

The product is the C-ABI library ``libsgagg.so`` (include/sgagg.h) built from
``csrc/``; ``sgagg`` is its Python binding.  Build with ``build.build()``.
"""
from . import build  # noqa: F401
from .sgagg import (Aggregator, SgaggError, sgagg_create, sgagg_destroy,  # noqa: F401
                    sgagg_aggregate, sgagg_aggregate_host, sgagg_aggregate_batched,
                    sgagg_result_rows, sgagg_temp_bytes, sgagg_stats, sgagg_last_error,
                    sgagg_set_option, SGAGG_COUNT, SGAGG_SUM, SGAGG_MIN, SGAGG_MAX)
