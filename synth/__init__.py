"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package holds no arithmetic of the embedding method: it only builds
graphs (R-MAT, Chakrabarti-Zhan-Faloutsos 2004; degree-corrected planted
partitions, Karrer-Newman 2011), their CSR form, and the
80/20 link-prediction split of Sec. 6.1.  The paper's datasets (SNAP,
WebDataCommons) are not available; these graphs stand in for them.
"""
from .rmat import (Graph, LinkSplit, rmat_edges, to_csr, rmat_graph, link_split,
                   random_graph, csr_from_edges, workload, fit_pairs, rmat_graph_large)
from .sbm import sbm_edges, sbm_graph

__all__ = ["Graph", "LinkSplit", "rmat_edges", "to_csr", "rmat_graph", "link_split",
           "random_graph", "csr_from_edges", "workload", "fit_pairs", "rmat_graph_large", "sbm_edges", "sbm_graph"]
