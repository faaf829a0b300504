"""dsr: a GB300 (sm_103a) SOA object allocator and parallel do-all (DynaSOAr, arXiv 1809.07444)."""
