// nrm_serve.cu placeholder
